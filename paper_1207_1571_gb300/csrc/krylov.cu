// krylov.cu -- persistent, cooperative Krylov solvers (paper Sec. 3:
// Jacobi-preconditioned CG for pressure, Jacobi-preconditioned BiCGStab for
// momentum; Sec. 4.3.2: SMVP, daxpy, dot product, reduction and diagonal
// preconditioner are the building blocks).
//
// One launch runs a whole solve.  The grid is sized to be co-resident
// (cooperative launch); phases are separated by a grid barrier that spins a
// bounded number of times and otherwise records FV_E_TIMEOUT.  Reductions
// are deterministic: each block writes its partial sums, and after the
// barrier every block adds all partials in the same fixed order, so every
// block takes the same decisions (convergence, breakdown) from bit-identical
// scalars.  Rows are owned by a fixed thread for the whole solve, so a
// thread only reads other threads' data where the algorithm needs neighbour
// values (matrix-vector products); the barrier's acquire orders those loads
// after the writes of the previous phase.  The same ownership lets the CG
// kernels keep their row-local vectors in shared memory for the whole solve
// where a block's rows fit (the resident forms, k_pcg<true> and
// k_pcg_mixed<true>).
//
// CG works on the symmetrically scaled system  D^-1/2 A D^-1/2 y = D^-1/2 b
// with x = D^-1/2 y: in exact arithmetic this generates the same iterates,
// step lengths and residual norms as Jacobi-preconditioned CG on A x = b
// (z = D^-1 r becomes the identity and r.z becomes r^.r^), while the product
// needs no diagonal and the preconditioner no extra pass.  The stopping test
// uses the unscaled residual ||r||_2 = ||D^1/2 r^||_2, exactly as the
// unscaled method does.
#include <cooperative_groups.h>

#include <cstdlib>
#include <cstring>

#include "fvgb_internal.h"
#include "coop.cuh"

namespace fvgb {

long long g_spin_limit = 1LL << 25;
constexpr int kBlock = 512;

struct RowSpan {
    int e0, K;
};

__device__ __forceinline__ RowSpan row_span(const int32_t *__restrict__ slice_ptr, int i)
{
    const int s = i >> 5;
    const int p0 = slice_ptr[s], p1 = slice_ptr[s + 1];
    return {p0 + (i & 31), (p1 - p0) >> 5};
}

// ------------------------------------------------------------ barriers --
// (grid barrier and deterministic reductions: coop.cuh)

// Sum v over the grid; every thread of every block returns the same bits
// (the reductions of coop.cuh: four warps per block in fixed trees, then one
// warp per value over the block partials).
constexpr int kBicgSums = 6;                // most values summed at once

__device__ __forceinline__ double (*bicg_sum_buffer())[kBlock]
{
    __shared__ double buf[kBicgSums][kBlock];   // one buffer for every NV
    return buf;
}

template <int NV>
__device__ bool grid_sum(double (&v)[NV], double *part, GridBar *bar, unsigned &gen, long long limit)
{
    static_assert(NV <= kBicgSums && NV <= kParts, "too many values");
    __shared__ double tot[NV];
    if (!cg_grid_sum<NV, kBlock>(v, part, bar, gen, limit, bicg_sum_buffer(), tot)) return false;
    if (gridDim.x == 1) __syncthreads();    // otherwise cg_grid_sum ended with one
#pragma unroll
    for (int k = 0; k < NV; ++k) v[k] = tot[k];
    return true;
}

// ------------------------------------------------------------------ CG --
//
// One block of kCgBlock threads per SM; block b owns the contiguous rows
// [b*chunk, (b+1)*chunk) (whole 32-row slices) for the whole solve, so the
// neighbour gathers of a block mostly hit its own SM's L1.  Gathers are
// plain loads: the grid barrier's acquire orders them after the writes of
// the previous phase.  Reductions run over four warps, one per SM
// sub-partition (coop.cuh).

struct CgArgs {
    int N;
    const int32_t *slice_ptr, *col;
    double *val;
    const double *diag, *b;
    double *x, *s, *r, *p, *q, *y;
    double *partA, *partB;
    GridBar *bar;
    long long spin;
    double tol, reltol;
    int maxit;
    DevSolveStats *stats;
};

// Scalar state of a CG solve, kept in shared memory and updated by thread 0
// only (one FP64 divide or square root costs a warp dozens of cycles per
// instruction on this part, so no thread repeats it).
struct CgScalars {
    double alpha, beta, rho, thresh, nb, nr0, nr, dmin;
    double near2;    // kNearStop thresh^2: evaluate the norm once min(D) r^.r^ is below it
    double skip2;    // thresh^2 kBoundMargin: a skipped evaluation could not stop above it
    double nrb2;     // min(D) r^.r^ of the last iteration when its norm was not evaluated
    int phase;       // 0 iterate, 1 converged, 2 not converged, 3 diverged, 4 zero rhs
    int exact;       // evaluate ||D^1/2 r^|| in this iteration's residual update
    int bound;       // the last iteration skipped the evaluation (nr = sqrt(nrb2), a lower bound)
};

// The stopping test needs ||r||_2 = ||D^1/2 r^||_2, two more FP64 operations
// per row than the r^.r^ the iteration needs anyway.  Since ||D^1/2 r^||^2 >=
// min(D) r^.r^, that norm is only evaluated once min(D) r^.r^ has come within
// kNearStop of thresh^2 (or at the iteration limit); if r^.r^ then falls past
// the bound in a single step, one extra pass evaluates it before the test.
// A skipped evaluation could not have met the test (the bound holds with a
// 1e-8 relative margin, far above the rounding of the sums), so iterates,
// counts and results are those of evaluating it every iteration.
constexpr double kNearStop = 16.0;
constexpr double kBoundMargin = 1.0 + 1e-8;

// Minimum over the block (all threads receive it).
__device__ __forceinline__ double block_min(double v)
{
    __shared__ double wmin[kCgBlock / 32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(0xffffffffu, v, o));
    if ((threadIdx.x & 31) == 0) wmin[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x < 32) {
        double w = threadIdx.x < (int)(blockDim.x >> 5) ? wmin[threadIdx.x] : INFINITY;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) w = fmin(w, __shfl_xor_sync(0xffffffffu, w, o));
        if (threadIdx.x == 0) wmin[0] = w;
    }
    __syncthreads();
    const double r = wmin[0];
    __syncthreads();
    return r;
}

// q = A^ p for one row of the unit-diagonal scaled matrix; all loads of
// the row are issued before the first product (rows have <= 6 entries on
// hexahedral and tetrahedral meshes; longer rows take the loop).
__device__ __forceinline__ double spmv_unit_row(const CgArgs &a, const RowSpan &rs, double pi)
{
    double acc = pi;
    if (rs.K <= 6) {
        int c[6];
        double v[6], x[6];
#pragma unroll
        for (int k = 0; k < 6; ++k)
            if (k < rs.K) { c[k] = a.col[rs.e0 + 32 * k]; v[k] = a.val[rs.e0 + 32 * k]; }
#pragma unroll
        for (int k = 0; k < 6; ++k)
            if (k < rs.K) x[k] = a.p[c[k]];
#pragma unroll
        for (int k = 0; k < 6; ++k)
            if (k < rs.K) acc += v[k] * x[k];
    } else {
        for (int k = 0; k < rs.K; ++k) {
            const int e = rs.e0 + 32 * k;
            acc += a.val[e] * a.p[a.col[e]];
        }
    }
    return acc;
}

// End of a CG iteration (thread 0): tot[0] = r^.r^, tot[1] = ||D^1/2 r^||^2
// when sc.exact != 0.  Takes the stopping decision, else beta, and whether
// the next iteration evaluates the norm.  The square root is only taken where
// the norm was evaluated; a skipped iteration keeps the lower bound
// min(D) r^.r^, which is finite whenever rho is.
__device__ __forceinline__ void cg_end_iteration(CgScalars &sc, const double *tot, int it, int maxit)
{
    const double rho = tot[0];
    const bool have = sc.exact != 0;
    if (have) sc.nr = sqrt(tot[1]);
    else sc.nrb2 = sc.dmin * rho;
    sc.bound = !have;
    if ((have && !isfinite(sc.nr)) || !isfinite(rho)) sc.phase = 3;
    else if (have && sc.nr <= sc.thresh) sc.phase = 1;
    else if (it >= maxit) sc.phase = 2;
    else {
        sc.beta = rho / sc.rho;
        sc.rho = rho;
        sc.exact = sc.dmin * rho <= sc.near2 ? 1 : 0;
    }
}

// Rows of block b: [b chunk, min(N, (b + 1) chunk)), whole 32-row slices.
__host__ __device__ __forceinline__ int cg_chunk(int N, int G)
{
    const int nsl = (N + 31) >> 5;
    return ((nsl + G - 1) / G) * 32;
}

// RES: the row-local vectors r^, q and y (each read and written only by the
// thread that owns the row) live in the block's shared memory, 3 x chunk
// doubles of dynamic shared memory; only p (gathered by neighbouring rows)
// and the matrix go through L2 and HBM.  On the 1M-cell cavity a block owns
// 6592 rows: 158 KB of the 227 KB a block may hold.  Otherwise the vectors
// are the workspace arrays in global memory.  Both forms do the same
// arithmetic in the same order.
template <bool RES>
__global__ void __launch_bounds__(kCgBlock, 1) k_pcg(CgArgs a)
{
    __shared__ double buf[3][kCgBlock];
    __shared__ double tot[3];
    __shared__ CgScalars sc;
    extern __shared__ double resv[];
    const int N = a.N;
    const int chunk = cg_chunk(N, gridDim.x);
    const int rb = blockIdx.x * chunk;
    const int nl = min(N, rb + chunk) - rb;      // rows of this block (none if <= 0)
    const int t0 = threadIdx.x;
    // own-row views, indexed by the row's offset in the block
    double *const rl = RES ? resv : a.r + rb;
    double *const ql = RES ? resv + chunk : a.q + rb;
    double *const yl = RES ? resv + 2 * chunk : a.y + rb;
    unsigned gen = 0;
    bool ok = true;
    int it = 0;

    // S1: scaling s = D^-1/2 and scaled start y = D^1/2 x; the block's
    // smallest diagonal (0 if any is not positive) in its partial record
    {
        double dmin = INFINITY;
        for (int l = t0; l < nl; l += kCgBlock) {
            const int i = rb + l;
            const double d = a.diag[i];
            const double sq = sqrt(d);
            a.s[i] = 1.0 / sq;
            yl[l] = a.x[i] * sq;
            dmin = d > 0.0 ? fmin(dmin, d) : 0.0;
        }
        dmin = block_min(dmin);
        if (threadIdx.x == 0) a.partA[blockIdx.x * kParts + kParts - 1] = dmin;
    }
    ok = grid_sync(a.bar, gen, a.spin);
    // S2: scale the off-diagonals, r^ = s (b - A x), norms
    if (ok) {
        double v3[3] = {0.0, 0.0, 0.0};   // ||b||^2, ||r||^2, r^.r^
        for (int l = t0; l < nl; l += kCgBlock) {
            const int i = rb + l;
            const RowSpan rs = row_span(a.slice_ptr, i);
            const double si = a.s[i], d = a.diag[i], xi = a.x[i];
            double ax = d * xi;
            for (int k = 0; k < rs.K; ++k) {
                const int e = rs.e0 + 32 * k;
                const int c = a.col[e];
                const double v = a.val[e];
                ax += v * a.x[c];
                a.val[e] = v * si * a.s[c];
            }
            const double bi = a.b[i];
            const double rh = si * (bi - ax);
            rl[l] = rh;
            v3[0] += bi * bi;
            v3[1] += d * rh * rh;
            v3[2] += rh * rh;
        }
        ok = cg_grid_sum<3>(v3, a.partB, a.bar, gen, a.spin, buf, tot);
    }
    if (threadIdx.x < 32) {
        // smallest diagonal over the grid (written before the last barrier)
        double m = INFINITY;
        for (int j = threadIdx.x; j < (int)gridDim.x; j += 32)
            m = fmin(m, __ldcg(a.partA + j * kParts + kParts - 1));
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) m = fmin(m, __shfl_xor_sync(0xffffffffu, m, o));
        if (threadIdx.x == 0) sc.dmin = m;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        sc.nb = sqrt(tot[0]);
        sc.nr0 = sqrt(tot[1]);
        sc.nr = sc.nr0;
        sc.rho = tot[2];
        sc.thresh = fmax(a.tol * sc.nb, a.reltol * sc.nr0);
        sc.near2 = kNearStop * sc.thresh * sc.thresh;
        sc.skip2 = (sc.thresh * sc.thresh) * kBoundMargin;
        sc.alpha = sc.beta = 0.0;
        sc.phase = sc.nb == 0.0 ? 4 : (sc.nr0 <= sc.thresh ? 1 : 0);
        sc.exact = 1;
        sc.bound = 0;
    }
    __syncthreads();
    if (ok && sc.phase == 4) {
        for (int l = t0; l < nl; l += kCgBlock) a.x[rb + l] = 0.0;
    } else if (ok && sc.phase == 0) {
        double *const pl = a.p + rb;
        while (true) {
            ++it;
            // P1: p = r^ + beta p (first: p = r^); y += alpha_prev p_prev
            if (it == 1) {
                for (int l = t0; l < nl; l += kCgBlock) pl[l] = rl[l];
            } else {
                // restrict-qualified copies and all three loads before the
                // two stores: several rows' loads stay in flight at once
                // (with y += alpha p written as a load-modify-store first,
                // this pass ran at 62 % of the copy bandwidth instead of 80 %)
                const double alpha = sc.alpha, beta = sc.beta;
                double *__restrict__ yv = yl;
                double *__restrict__ pv = pl;
                const double *__restrict__ rv = rl;
#pragma unroll 4
                for (int l = t0; l < nl; l += kCgBlock) {
                    const double po = pv[l];
                    const double ri = rv[l];
                    const double yi = yv[l];
                    pv[l] = ri + beta * po;
                    yv[l] = yi + alpha * po;
                }
            }
            if (!(ok = grid_sync(a.bar, gen, a.spin))) break;
            // P2: q = A^ p (unit diagonal), p.q
            double v1[1] = {0.0};
            {
                double *__restrict__ qv = ql;
#pragma unroll 2
                for (int l = t0; l < nl; l += kCgBlock) {
                    const int i = rb + l;
                    const RowSpan rs = row_span(a.slice_ptr, i);
                    const double pi = a.p[i];
                    const double acc = spmv_unit_row(a, rs, pi);
                    qv[l] = acc;
                    v1[0] += pi * acc;
                }
            }
            if (!(ok = cg_grid_sum<1>(v1, a.partA, a.bar, gen, a.spin, buf, tot))) break;
            if (threadIdx.x == 0) {
                const double pq = tot[0];
                if (!(pq > 0.0) || !isfinite(pq)) { sc.phase = 3; sc.alpha = 0.0; }
                else sc.alpha = sc.rho / pq;
            }
            __syncthreads();
            if (sc.phase == 3) break;
            // P3: r^ -= alpha q; r^.r^, and ||D^1/2 r^||^2 near the stop
            const double alpha = sc.alpha;
            const bool exact = sc.exact || it >= a.maxit;
            {
                double *__restrict__ rv = rl;
                const double *__restrict__ qv = ql;
                const double *__restrict__ dv = a.diag + rb;
                if (exact) {
                    double v2[2] = {0.0, 0.0};
                    for (int l = t0; l < nl; l += kCgBlock) {
                        const double ri = rv[l] - alpha * qv[l];
                        rv[l] = ri;
                        v2[0] += ri * ri;
                        v2[1] += (dv[l] * ri) * ri;
                    }
                    ok = cg_grid_sum<2>(v2, a.partB, a.bar, gen, a.spin, buf, tot);
                } else {
                    // the common case, a tight loop (a uniform branch inside the
                    // unrolled loop cost a third of this pass's bandwidth) and a
                    // sum of one value (each FP64 value summed over the block
                    // costs a few hundred cycles)
                    double v1[1] = {0.0};
#pragma unroll 4
                    for (int l = t0; l < nl; l += kCgBlock) {
                        const double ri = rv[l] - alpha * qv[l];
                        rv[l] = ri;
                        v1[0] += ri * ri;
                    }
                    ok = cg_grid_sum<1>(v1, a.partB, a.bar, gen, a.spin, buf, tot);
                }
            }
            if (!ok) break;
            if (threadIdx.x == 0) {
                // an evaluation skipped while the bound still allows the stop
                sc.exact = exact ? 1 : (sc.dmin * tot[0] > sc.skip2 ? 0 : 2);
                if (sc.exact != 2) cg_end_iteration(sc, tot, it, a.maxit);
            }
            __syncthreads();
            if (sc.exact == 2) {
                double v4[1] = {0.0};
                for (int l = t0; l < nl; l += kCgBlock) {
                    const double ri = rl[l];
                    v4[0] += (a.diag[rb + l] * ri) * ri;
                }
                if (!(ok = cg_grid_sum<1>(v4, a.partA, a.bar, gen, a.spin, buf, tot + 1))) break;
                if (threadIdx.x == 0) cg_end_iteration(sc, tot, it, a.maxit);
                __syncthreads();
            }
            if (sc.phase != 0) break;
        }
        if (ok) {
            // final update of the scaled iterate, then x = D^-1/2 y
            const double af = (sc.phase == 3) ? 0.0 : sc.alpha;
            for (int l = t0; l < nl; l += kCgBlock) {
                const int i = rb + l;
                a.x[i] = a.s[i] * (yl[l] + af * a.p[i]);
            }
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        const int ph = sc.phase;
        a.stats->iters = it;
        a.stats->status = !ok ? FV_E_TIMEOUT
                        : ph == 3 ? FV_E_DIVERGED : ph == 2 ? FV_E_NOT_CONVERGED : FV_OK;
        const bool zero = ph == 4;
        a.stats->res0 = zero ? 0.0 : sc.nr0 / sc.nb;
        const double nr = sc.bound ? sqrt(sc.nrb2) : sc.nr;
        a.stats->res = zero ? 0.0 : nr / sc.nb;
        a.stats->outer = 1;
    }
}

// ------------------------------------------------------ mixed precision --
//
// FP32 Jacobi-CG with reliable updates and one deflation vector, inside FP64
// defect correction (not in the paper, whose Fermi code is FP64 throughout).
//
// * FP64: the true residual r = b - A x with the FP64 matrix, its norm, the
//   stopping test ||b - A x|| <= max(tol ||b||, reltol ||r0||), the solution
//   x, and all reductions across threads and blocks.
// * FP32: the CG recurrences (p, q, r^ and the correction e) on an FP32 copy
//   of the symmetrically scaled matrix A^ = D^-1/2 A D^-1/2; products are
//   summed in FP32 over a thread's rows.
// * Reliable updates: when the FP32 residual has fallen by kReliable since the
//   last refresh, or predicts convergence, or p.A^p is not positive, e is
//   folded into x and the residual is recomputed in FP64; the search
//   direction is kept (restarted only after a non-positive curvature).
// * Deflation: a pressure matrix pinned at one reference cell (closed
//   domains) has one eigenvalue of order 1/N (the constant mode), which FP32
//   CG cannot resolve.  Search directions are kept A^-orthogonal to
//   w = D^1/2 1 (p = r^ + beta p - w (v.r^)/mu with v = A^ w = D^-1/2 A 1,
//   mu = 1.A.1) and every refresh first removes the residual's component
//   along the mode with the constant shift x += (1.r)/mu.

constexpr double kReliable = 0.1;

struct MixArgs {
    int N;
    const int32_t *slice_ptr, *col;
    const double *val;      // FP64 off-diagonals (unscaled), read only
    float *val32;           // FP32 scaled off-diagonals (written in setup)
    const double *diag, *b;
    double *x, *s, *r64, *a1;
    float *r, *p, *q, *e, *w, *v;
    double *partA, *partB;
    GridBar *bar;
    long long spin;
    double tol, reltol;
    int maxit;
    DevSolveStats *stats;
};

struct MixScalars {
    double nb, nr0, nr, thresh, rho, rho_ref, ratio, alpha, beta, mu, delta, shift;
    double inv_mu;   // 1 / mu (the deflation coefficient of every inner iteration)
    double rel2;     // kReliable^2 rho_ref: refresh once r^.r^ falls below it
    double pred2;    // (thresh / ratio)^2: r^.r^ below it predicts convergence
    int phase;       // 0 run, 1 converged, 2 iteration budget used, 3 breakdown, 4 zero rhs
    int refresh;     // 1: refresh after this iteration, 2: refresh and restart p
    int restart;     // restart the search direction at the next iteration
    int bad;         // consecutive forced refreshes without progress
    int deflate;
};

__device__ __forceinline__ float spmv32_unit_row(const MixArgs &a, const RowSpan &rs, float pi)
{
    float acc = pi;
    if (rs.K <= 6) {
        int c[6];
        float v[6], x[6];
#pragma unroll
        for (int k = 0; k < 6; ++k)
            if (k < rs.K) { c[k] = a.col[rs.e0 + 32 * k]; v[k] = a.val32[rs.e0 + 32 * k]; }
#pragma unroll
        for (int k = 0; k < 6; ++k)
            if (k < rs.K) x[k] = a.p[c[k]];
#pragma unroll
        for (int k = 0; k < 6; ++k)
            if (k < rs.K) acc = fmaf(v[k], x[k], acc);
    } else {
        for (int k = 0; k < rs.K; ++k) {
            const int e = rs.e0 + 32 * k;
            acc = fmaf(a.val32[e], a.p[a.col[e]], acc);
        }
    }
    return acc;
}

// Rows i and i + 1 (i even) of the FP32 scaled matrix: they share a SELL
// slice and sit in adjacent slots, so one 8-byte load brings both rows'
// columns and both values of a slot.  The global form of k_pcg_mixed works
// on row pairs this way: its passes stream from HBM, and with 4-byte loads
// a thread keeps half the bytes in flight that the FP64 CG's 8-byte loads
// do (8M cavity: 184 -> 163 us per inner iteration).  The resident form
// keeps one row per thread (with pairs its L2- and latency-bound passes ran
// slower: 18.0 -> 21.9 us per inner iteration on the 1M cavity).
__device__ __forceinline__ float2 spmv32_unit_pair(const MixArgs &a, const RowSpan &rs, float2 pi)
{
    float2 acc = pi;
#pragma unroll 6
    for (int k = 0; k < rs.K; ++k) {
        const int e = rs.e0 + 32 * k;
        const int2 c = *reinterpret_cast<const int2 *>(a.col + e);
        const float2 v = *reinterpret_cast<const float2 *>(a.val32 + e);
        acc.x = fmaf(v.x, a.p[c.x], acc.x);
        acc.y = fmaf(v.y, a.p[c.y], acc.y);
    }
    return acc;
}

// RES: the row-local FP32 vectors r^, q, e, w and v (each read and written
// only by the thread that owns the row) live in the block's shared memory,
// 5 x chunk floats of dynamic shared memory; p (gathered by neighbouring
// rows), the matrices and the FP64 vectors stay in global memory.  The global
// form takes two neighbouring rows per thread in its inner passes (8-byte
// accesses), which groups the per-thread sums differently from the resident
// form.
template <bool RES>
__global__ void __launch_bounds__(kCgBlock, 1) k_pcg_mixed(MixArgs a)
{
    __shared__ double buf[3][kCgBlock];
    __shared__ double tot[3];
    __shared__ MixScalars sc;
    const int N = a.N;
    const int nsl = (N + 31) >> 5;
    const int chunk = ((nsl + gridDim.x - 1) / gridDim.x) * 32;
    const int rb = blockIdx.x * chunk;
    const int re = min(N, rb + chunk);
    const int i0 = rb + threadIdx.x;
    const int ip = rb + 2 * (int)threadIdx.x;     // global form: first row of this thread's pairs
    extern __shared__ float resf[];
    // the FP32 row vectors, indexed by i - o: shared (offset by the block's
    // first row) or global
    const int o = RES ? rb : 0;
    float *const rl = RES ? resf : a.r;
    float *const ql = RES ? resf + chunk : a.q;
    float *const el = RES ? resf + 2 * chunk : a.e;
    float *const wl = RES ? resf + 3 * chunk : a.w;
    float *const vl = RES ? resf + 4 * chunk : a.v;
    unsigned gen = 0;
    bool ok = true;
    int it = 0, outer = 0;

    // S1: scaling
    for (int i = i0; i < re; i += kCgBlock) a.s[i] = 1.0 / sqrt(a.diag[i]);
    ok = grid_sync(a.bar, gen, a.spin);
    // S2: FP32 scaled matrix, A 1 (FP64), w = D^1/2 1, v = D^-1/2 A 1, mu = 1.A.1
    if (ok) {
        double v1[1] = {0.0};
        for (int i = i0; i < re; i += kCgBlock) {
            const RowSpan rs = row_span(a.slice_ptr, i);
            const double si = a.s[i];
            double row = a.diag[i];
            for (int k = 0; k < rs.K; ++k) {
                const int e = rs.e0 + 32 * k;
                const double v = a.val[e];
                row += v;
                a.val32[e] = (float)(v * si * a.s[a.col[e]]);
            }
            a.a1[i] = row;
            wl[i - o] = (float)(1.0 / si);
            vl[i - o] = (float)(si * row);
            v1[0] += row;
        }
        ok = cg_grid_sum<1>(v1, a.partA, a.bar, gen, a.spin, buf, tot);
    }
    if (threadIdx.x == 0) {
        sc.phase = 0;
        sc.alpha = sc.beta = sc.delta = 0.0;
        sc.restart = 1;
        sc.bad = 0;
        sc.refresh = 0;
        sc.nr = 0.0;
        sc.mu = tot[0];
        sc.inv_mu = 1.0 / tot[0];
        sc.deflate = (tot[0] > 0.0 && isfinite(tot[0])) ? 1 : 0;
    }
    __syncthreads();
    while (ok) {
        // R1: FP64 true residual from x; 1.r for the coarse correction
        double v2[2] = {0.0, 0.0};     // ||b||^2, 1.r
        for (int i = i0; i < re; i += kCgBlock) {
            const RowSpan rs = row_span(a.slice_ptr, i);
            double ax = a.diag[i] * a.x[i];
            for (int k = 0; k < rs.K; ++k) {
                const int e = rs.e0 + 32 * k;
                ax += a.val[e] * a.x[a.col[e]];
            }
            const double bi = a.b[i];
            const double ri = bi - ax;
            a.r64[i] = ri;
            v2[0] += bi * bi;
            v2[1] += ri;
        }
        if (!(ok = cg_grid_sum<2>(v2, a.partB, a.bar, gen, a.spin, buf, tot))) break;
        if (threadIdx.x == 0) {
            if (outer == 0) sc.nb = sqrt(tot[0]);
            sc.shift = sc.deflate ? tot[1] / sc.mu : 0.0;
        }
        __syncthreads();
        // R2: coarse correction x += shift (r -= shift A 1), FP32 scaled residual
        {
            const double sh = sc.shift;
            double v3[3] = {0.0, 0.0, 0.0};     // ||r||^2, r^.r^, v.r^
            for (int i = i0; i < re; i += kCgBlock) {
                const double ri = a.r64[i] - sh * a.a1[i];
                a.x[i] += sh;
                const float rh = (float)(a.s[i] * ri);
                rl[i - o] = rh;
                el[i - o] = 0.0f;
                v3[0] += ri * ri;
                v3[1] += (double)rh * (double)rh;
                v3[2] += (double)vl[i - o] * (double)rh;
            }
            if (!(ok = cg_grid_sum<3>(v3, a.partA, a.bar, gen, a.spin, buf, tot))) break;
        }
        if (threadIdx.x == 0) {
            const double prev = sc.nr;
            sc.nr = sqrt(tot[0]);
            if (outer == 0) {
                sc.nr0 = sc.nr;
                sc.thresh = fmax(a.tol * sc.nb, a.reltol * sc.nr0);
                if (sc.nb == 0.0) sc.phase = 4;
            } else if (sc.refresh == 2) {
                sc.bad = (sc.nr >= prev) ? sc.bad + 1 : 0;
                if (sc.bad >= 2) sc.phase = 3;
            }
            if (sc.phase == 0) {
                if (!isfinite(sc.nr)) sc.phase = 3;
                else if (sc.nr <= sc.thresh) sc.phase = 1;
                else if (it >= a.maxit) sc.phase = 2;
            }
            // continue CG with the refreshed residual (van der Vorst - Ye)
            sc.beta = (outer > 0 && sc.restart == 0 && sc.rho > 0.0) ? tot[1] / sc.rho : 0.0;
            sc.rho = tot[1];
            sc.rho_ref = tot[1];
            sc.ratio = tot[1] > 0.0 ? sc.nr / sqrt(tot[1]) : 0.0;
            // the inner iterations compare r^.r^ with squared thresholds (a
            // square root and a divide on thread 0 per iteration saved)
            sc.rel2 = kReliable * kReliable * sc.rho_ref;
            sc.pred2 = sc.ratio > 0.0 ? (sc.thresh / sc.ratio) * (sc.thresh / sc.ratio) : INFINITY;
            sc.delta = sc.deflate ? tot[2] / sc.mu : 0.0;
            sc.alpha = 0.0;          // the correction was folded into x
            sc.refresh = 0;
        }
        __syncthreads();
        ++outer;
        if (sc.phase != 0) break;
        // FP32 CG iterations until the next refresh
        while (true) {
            ++it;
            const float alpha = (float)sc.alpha, beta = (float)sc.beta, delta = (float)sc.delta;
            if (sc.restart) {
                for (int i = i0; i < re; i += kCgBlock) a.p[i] = fmaf(-delta, wl[i - o], rl[i - o]);
            } else if (RES) {
                // all loads before the stores (as in the FP64 CG)
                float *__restrict__ pv = a.p;
                float *__restrict__ ev = el;
                const float *__restrict__ rv = rl;
                const float *__restrict__ wv = wl;
#pragma unroll 4
                for (int i = i0; i < re; i += kCgBlock) {
                    const float po = pv[i], ei = ev[i - o], ri = rv[i - o], wi = wv[i - o];
                    ev[i - o] = fmaf(alpha, po, ei);
                    pv[i] = fmaf(-delta, wi, fmaf(beta, po, ri));
                }
            } else {
                // global form: row pairs with 8-byte accesses, all loads before
                // the stores; an odd last row alone
                float *__restrict__ pv = a.p;
                float *__restrict__ ev = el;
                const float *__restrict__ rv = rl;
                const float *__restrict__ wv = wl;
#pragma unroll 2
                for (int i = ip; i < re; i += 2 * kCgBlock) {
                    if (i + 1 < re) {
                        const float2 po = *reinterpret_cast<const float2 *>(pv + i);
                        const float2 ei = *reinterpret_cast<const float2 *>(ev + i);
                        const float2 ri = *reinterpret_cast<const float2 *>(rv + i);
                        const float2 wi = *reinterpret_cast<const float2 *>(wv + i);
                        *reinterpret_cast<float2 *>(ev + i) =
                            make_float2(fmaf(alpha, po.x, ei.x), fmaf(alpha, po.y, ei.y));
                        *reinterpret_cast<float2 *>(pv + i) =
                            make_float2(fmaf(-delta, wi.x, fmaf(beta, po.x, ri.x)),
                                        fmaf(-delta, wi.y, fmaf(beta, po.y, ri.y)));
                    } else {
                        const float po = pv[i], ei = ev[i], ri = rv[i], wi = wv[i];
                        ev[i] = fmaf(alpha, po, ei);
                        pv[i] = fmaf(-delta, wi, fmaf(beta, po, ri));
                    }
                }
            }
            if (!(ok = grid_sync(a.bar, gen, a.spin))) break;
            float pq32 = 0.0f;
            if (RES) {
#pragma unroll 2
                for (int i = i0; i < re; i += kCgBlock) {
                    const RowSpan rs = row_span(a.slice_ptr, i);
                    const float pi = a.p[i];
                    const float acc = spmv32_unit_row(a, rs, pi);
                    ql[i - o] = acc;
                    pq32 = fmaf(pi, acc, pq32);
                }
            } else {
                for (int i = ip; i < re; i += 2 * kCgBlock) {
                    const RowSpan rs = row_span(a.slice_ptr, i);
                    if (i + 1 < re) {
                        const float2 pi = *reinterpret_cast<const float2 *>(a.p + i);
                        const float2 acc = spmv32_unit_pair(a, rs, pi);
                        *reinterpret_cast<float2 *>(ql + i) = acc;
                        pq32 = fmaf(pi.x, acc.x, pq32);
                        pq32 = fmaf(pi.y, acc.y, pq32);
                    } else {
                        const float pi = a.p[i];
                        const float acc = spmv32_unit_row(a, rs, pi);
                        ql[i] = acc;
                        pq32 = fmaf(pi, acc, pq32);
                    }
                }
            }
            double v1[1] = {(double)pq32};
            if (!(ok = cg_grid_sum<1>(v1, a.partA, a.bar, gen, a.spin, buf, tot))) break;
            if (threadIdx.x == 0) {
                sc.restart = 0;
                const double pq = tot[0];
                if (!(pq > 0.0) || !isfinite(pq)) { sc.refresh = 2; sc.alpha = 0.0; }
                else sc.alpha = sc.rho / pq;
            }
            __syncthreads();
            if (sc.refresh == 2) break;
            const float al = (float)sc.alpha;
            float rr32 = 0.0f, vr32 = 0.0f;
            {
                float *__restrict__ rv = rl;
                const float *__restrict__ qv = ql;
                const float *__restrict__ vv = vl;
                if (RES) {
#pragma unroll 4
                    for (int i = i0; i < re; i += kCgBlock) {
                        const float qi = qv[i - o], rio = rv[i - o], vi = vv[i - o];
                        const float ri = fmaf(-al, qi, rio);
                        rv[i - o] = ri;
                        rr32 = fmaf(ri, ri, rr32);
                        vr32 = fmaf(vi, ri, vr32);
                    }
                } else {
#pragma unroll 2
                    for (int i = ip; i < re; i += 2 * kCgBlock) {
                        if (i + 1 < re) {
                            const float2 qi = *reinterpret_cast<const float2 *>(qv + i);
                            const float2 rio = *reinterpret_cast<const float2 *>(rv + i);
                            const float2 vi = *reinterpret_cast<const float2 *>(vv + i);
                            const float r0 = fmaf(-al, qi.x, rio.x), r1 = fmaf(-al, qi.y, rio.y);
                            *reinterpret_cast<float2 *>(rv + i) = make_float2(r0, r1);
                            rr32 = fmaf(r0, r0, rr32);
                            rr32 = fmaf(r1, r1, rr32);
                            vr32 = fmaf(vi.x, r0, vr32);
                            vr32 = fmaf(vi.y, r1, vr32);
                        } else {
                            const float qi = qv[i], rio = rv[i], vi = vv[i];
                            const float ri = fmaf(-al, qi, rio);
                            rv[i] = ri;
                            rr32 = fmaf(ri, ri, rr32);
                            vr32 = fmaf(vi, ri, vr32);
                        }
                    }
                }
            }
            double v2[2] = {(double)rr32, (double)vr32};
            if (!(ok = cg_grid_sum<2>(v2, a.partB, a.bar, gen, a.spin, buf, tot))) break;
            if (threadIdx.x == 0) {
                const double rn = tot[0];
                if (!isfinite(rn)) { sc.refresh = 2; }
                else if (rn <= sc.rel2 || rn <= sc.pred2 || it >= a.maxit) {
                    // refresh; sc.rho keeps r.r of the previous iteration so
                    // that beta can be formed with the refreshed residual
                    sc.refresh = 1;
                } else {
                    sc.beta = rn / sc.rho;
                    sc.rho = rn;
                    sc.delta = sc.deflate ? tot[1] * sc.inv_mu : 0.0;
                }
            }
            __syncthreads();
            if (sc.refresh) break;
        }
        if (!ok) break;
        // fold the FP32 correction (with the last step) into the FP64 solution
        {
            const float al = (float)sc.alpha;
            for (int i = i0; i < re; i += kCgBlock) {
                const float ei = fmaf(al, a.p[i], el[i - o]);
                a.x[i] += a.s[i] * (double)ei;
            }
        }
        if (threadIdx.x == 0 && sc.refresh == 2) sc.restart = 1;
        __syncthreads();
        if (!(ok = grid_sync(a.bar, gen, a.spin))) break;
    }
    if (ok && sc.phase == 4)
        for (int i = i0; i < re; i += kCgBlock) a.x[i] = 0.0;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        const int ph = sc.phase;
        a.stats->iters = it;
        a.stats->status = !ok ? FV_E_TIMEOUT
                        : ph == 3 ? FV_E_DIVERGED : ph == 2 ? FV_E_NOT_CONVERGED : FV_OK;
        const bool zero = ph == 4;
        a.stats->res0 = zero ? 0.0 : sc.nr0 / sc.nb;
        a.stats->res = zero ? 0.0 : sc.nr / sc.nb;
        a.stats->outer = outer;
    }
}

// ----------------------------- mixed precision, Chronopoulos-Gear order --
//
// The same method (FP32 deflated CG with reliable updates inside FP64 defect
// correction) with the inner iterations in the order of Chronopoulos and
// Gear (1989): the product of an iteration is w = A^ r^ of the new
// residual, and with s = A^ p carried by the recurrence s = w + beta s the
// sums the next iteration needs -- r^.r^, w.r^ and, for the deflation,
// v.r^ -- are all formed with that product.  An iteration is then one
// vector pass, a grid barrier (the product gathers the neighbours' new
// residual) and one product pass ending in one grid sum: two
// synchronisations against three for the textbook order (k_pcg_mixed).
// (The fully pipelined order of Ghysels and Vanroose, one synchronisation
// with z = A^ s carried as well, broke down in FP32 on these pressure
// systems from 64^3 cells up, with or without replacing s and z at every
// reliable update; this order converges like the textbook one.)
//
// With c = (v.r^)/mu the deflated direction p = r^ + beta p - c w_d (w_d =
// D^1/2 1) has s = w + beta s - c v, and its curvature is
// p.A^p = w.r^ - beta r^.r^ / alpha_prev - (v.r^) c (the identities
// r^_k . r^_(k-1) = 0 and p_(k-1).A^p_k = 0).  After a reliable update the
// residual is the refreshed one, for which those identities hold only
// approximately, so that iteration takes its curvature from explicit sums
// (r^.s and p.s of the kept direction).  FP64 keeps the true residual, the
// stopping test, the solution and all cross-thread sums, as in k_pcg_mixed.

struct CgcgArgs {
    int N;
    const int32_t *slice_ptr, *col;
    const double *val;      // FP64 off-diagonals (unscaled), read only
    float *val32;           // FP32 scaled off-diagonals (written in setup)
    const double *diag, *b;
    double *x, *s64, *r64, *a1;
    float *r;                           // residual (global: gathered by neighbours)
    float *p, *sv, *e, *w;              // row-local (shared memory in the resident form)
    float *wd, *v;                      // deflation: w_d = D^1/2 1, v = A^ w_d
    double *partA, *partB;
    GridBar *bar;
    long long spin;
    double tol, reltol;
    int maxit;
    DevSolveStats *stats;
};

struct CgcgScalars {
    double nb, nr0, nr, thresh, rho, ratio, alpha, beta, c, mu, inv_mu, shift;
    double rel2, pred2;
    int phase;       // 0 run, 1 converged, 2 iteration budget used, 3 breakdown, 4 zero rhs
    int refresh;     // 1: refresh after this iteration, 2: refresh and restart p
    int restart;     // no kept search direction (first pass or after a breakdown)
    int bad;         // consecutive forced refreshes without progress
    int deflate;
};

__device__ __forceinline__ float spmv32_gather(const CgcgArgs &a, const RowSpan &rs,
                                               const float *__restrict__ src, float own)
{
    float acc = own;
    if (rs.K <= 6) {
        int c[6];
        float v[6], x[6];
#pragma unroll
        for (int k = 0; k < 6; ++k)
            if (k < rs.K) { c[k] = a.col[rs.e0 + 32 * k]; v[k] = a.val32[rs.e0 + 32 * k]; }
#pragma unroll
        for (int k = 0; k < 6; ++k)
            if (k < rs.K) x[k] = src[c[k]];
#pragma unroll
        for (int k = 0; k < 6; ++k)
            if (k < rs.K) acc = fmaf(v[k], x[k], acc);
    } else {
        for (int k = 0; k < rs.K; ++k) {
            const int e = rs.e0 + 32 * k;
            acc = fmaf(a.val32[e], src[a.col[e]], acc);
        }
    }
    return acc;
}

// RES: p, s, e and w (read and written only by the thread owning the row)
// live in the block's shared memory, 4 x chunk floats.
template <bool RES>
__global__ void __launch_bounds__(kCgBlock, 1) k_pcg_mixed_cgcg(CgcgArgs a)
{
    __shared__ double buf[5][kCgBlock];
    __shared__ double tot[5];
    __shared__ CgcgScalars sc;
    const int N = a.N;
    const int nsl = (N + 31) >> 5;
    const int chunk = ((nsl + gridDim.x - 1) / gridDim.x) * 32;
    const int rb = blockIdx.x * chunk;
    const int re = min(N, rb + chunk);
    const int i0 = rb + threadIdx.x;
    extern __shared__ float resc[];
    const int o = RES ? rb : 0;
    float *const pl = RES ? resc : a.p;
    float *const sl = RES ? resc + chunk : a.sv;
    float *const el = RES ? resc + 2 * chunk : a.e;
    float *const wl = RES ? resc + 3 * chunk : a.w;
    float *const rg = a.r;
    unsigned gen = 0;
    unsigned nred = 0;           // reductions so far: alternate partial buffers
    bool ok = true;
    int it = 0, outer = 0;
#define CGCG_PART (((nred++) & 1u) ? a.partB : a.partA)

    // S1: scaling
    for (int i = i0; i < re; i += kCgBlock) a.s64[i] = 1.0 / sqrt(a.diag[i]);
    ok = grid_sync(a.bar, gen, a.spin);
    // S2: FP32 scaled matrix, A 1 (FP64), w_d = D^1/2 1, v = D^-1/2 A 1, mu = 1.A.1
    if (ok) {
        double v1[1] = {0.0};
        for (int i = i0; i < re; i += kCgBlock) {
            const RowSpan rs = row_span(a.slice_ptr, i);
            const double si = a.s64[i];
            double row = a.diag[i];
            for (int k = 0; k < rs.K; ++k) {
                const int e = rs.e0 + 32 * k;
                const double v = a.val[e];
                row += v;
                a.val32[e] = (float)(v * si * a.s64[a.col[e]]);
            }
            a.a1[i] = row;
            a.wd[i] = (float)(1.0 / si);
            a.v[i] = (float)(si * row);
            v1[0] += row;
        }
        ok = cg_grid_sum<1>(v1, CGCG_PART, a.bar, gen, a.spin, buf, tot);
    }
    if (threadIdx.x == 0) {
        sc.phase = 0;
        sc.alpha = sc.beta = sc.c = 0.0;
        sc.restart = 1;
        sc.bad = 0;
        sc.refresh = 0;
        sc.nr = 0.0;
        sc.rho = 0.0;
        sc.mu = tot[0];
        sc.inv_mu = 1.0 / tot[0];
        sc.deflate = (tot[0] > 0.0 && isfinite(tot[0])) ? 1 : 0;
    }
    __syncthreads();
    while (ok) {
        // R1: FP64 true residual from x; 1.r for the coarse correction
        double v2[2] = {0.0, 0.0};     // ||b||^2, 1.r
        for (int i = i0; i < re; i += kCgBlock) {
            const RowSpan rs = row_span(a.slice_ptr, i);
            double ax = a.diag[i] * a.x[i];
            for (int k = 0; k < rs.K; ++k) {
                const int e = rs.e0 + 32 * k;
                ax += a.val[e] * a.x[a.col[e]];
            }
            const double bi = a.b[i];
            const double ri = bi - ax;
            a.r64[i] = ri;
            v2[0] += bi * bi;
            v2[1] += ri;
        }
        if (!(ok = cg_grid_sum<2>(v2, CGCG_PART, a.bar, gen, a.spin, buf, tot))) break;
        if (threadIdx.x == 0) {
            if (outer == 0) sc.nb = sqrt(tot[0]);
            sc.shift = sc.deflate ? tot[1] / sc.mu : 0.0;
        }
        __syncthreads();
        // R2: coarse correction x += shift, FP32 scaled residual, e = 0;
        // ||r||^2 in FP64
        {
            const double sh = sc.shift;
            double v1[1] = {0.0};
            for (int i = i0; i < re; i += kCgBlock) {
                const double ri = a.r64[i] - sh * a.a1[i];
                a.x[i] += sh;
                rg[i] = (float)(a.s64[i] * ri);
                el[i - o] = 0.0f;
                v1[0] += ri * ri;
            }
            if (!(ok = cg_grid_sum<1>(v1, CGCG_PART, a.bar, gen, a.spin, buf, tot))) break;
        }
        if (threadIdx.x == 0) {
            const double prev = sc.nr;
            sc.nr = sqrt(tot[0]);
            if (outer == 0) {
                sc.nr0 = sc.nr;
                sc.thresh = fmax(a.tol * sc.nb, a.reltol * sc.nr0);
                if (sc.nb == 0.0) sc.phase = 4;
            } else if (sc.refresh == 2) {
                sc.bad = (sc.nr >= prev) ? sc.bad + 1 : 0;
                if (sc.bad >= 2) sc.phase = 3;
            }
            if (sc.phase == 0) {
                if (!isfinite(sc.nr)) sc.phase = 3;
                else if (sc.nr <= sc.thresh) sc.phase = 1;
                else if (it >= a.maxit) sc.phase = 2;
            }
        }
        __syncthreads();
        ++outer;
        if (sc.phase != 0) break;
        // R3: w = A^ r^; the sums that start the iterations: r^.r^, w.r^, v.r^
        // and, for a kept direction, r^.s and p.s (else p = s = 0)
        {
            const bool keep = !sc.restart;
            float g = 0.0f, d = 0.0f, ep = 0.0f, sg = 0.0f, pp = 0.0f;
            for (int i = i0; i < re; i += kCgBlock) {
                const RowSpan rs = row_span(a.slice_ptr, i);
                const float ri = rg[i];
                const float wi = spmv32_gather(a, rs, rg, ri);
                wl[i - o] = wi;
                g = fmaf(ri, ri, g);
                d = fmaf(wi, ri, d);
                ep = fmaf(a.v[i], ri, ep);
                if (keep) {
                    const float si = sl[i - o];
                    sg = fmaf(ri, si, sg);
                    pp = fmaf(pl[i - o], si, pp);
                } else {
                    pl[i - o] = 0.0f;
                    sl[i - o] = 0.0f;
                }
            }
            double v5[5] = {(double)g, (double)d, (double)ep, (double)sg, (double)pp};
            if (!(ok = cg_grid_sum<5>(v5, CGCG_PART, a.bar, gen, a.spin, buf, tot))) break;
        }
        if (threadIdx.x == 0) {
            const double gam = tot[0], del = tot[1], eps = tot[2];
            const double c = sc.deflate ? eps * sc.inv_mu : 0.0;
            double beta = (!sc.restart && sc.rho > 0.0) ? gam / sc.rho : 0.0;
            // curvature of the new direction from explicit sums
            double den = del + beta * (2.0 * tot[3] + beta * tot[4]) - eps * c;
            if (!(den > 0.0) && beta != 0.0) {
                // drop the kept direction (p = s = 0 is not set here: beta = 0
                // multiplies them, and they are finite)
                beta = 0.0;
                den = del - eps * c;
            }
            if (!(den > 0.0) || !isfinite(den) || !isfinite(gam)) {
                sc.phase = 3;
            } else {
                sc.beta = beta;
                sc.c = c;
                sc.alpha = gam / den;
                sc.rho = gam;
                sc.ratio = gam > 0.0 ? sc.nr / sqrt(gam) : 0.0;
                sc.rel2 = kReliable * kReliable * gam;
                sc.pred2 = sc.ratio > 0.0 ? (sc.thresh / sc.ratio) * (sc.thresh / sc.ratio) : INFINITY;
                sc.refresh = 0;
                sc.restart = 0;
            }
        }
        __syncthreads();
        if (sc.phase != 0) break;
        // inner iterations: a vector pass, a barrier, the product with its sum
        while (true) {
            ++it;
            {
                const float al = (float)sc.alpha, be = (float)sc.beta, cc = (float)sc.c;
                float *__restrict__ pv = pl;
                float *__restrict__ sv = sl;
                float *__restrict__ ev = el;
                float *__restrict__ rv = rg;
                const float *__restrict__ wv = wl;
#pragma unroll 2
                for (int i = i0; i < re; i += kCgBlock) {
                    const float po = pv[i - o], so = sv[i - o], eo = ev[i - o];
                    const float ri = rv[i], wi = wv[i - o], wdi = a.wd[i], vi = a.v[i];
                    const float pi = fmaf(-cc, wdi, fmaf(be, po, ri));
                    const float si = fmaf(-cc, vi, fmaf(be, so, wi));
                    pv[i - o] = pi;
                    sv[i - o] = si;
                    ev[i - o] = fmaf(al, pi, eo);
                    rv[i] = fmaf(-al, si, ri);
                }
            }
            if (!(ok = grid_sync(a.bar, gen, a.spin))) break;
            float g = 0.0f, d = 0.0f, ep = 0.0f;
            {
                float *__restrict__ wv = wl;
#pragma unroll 2
                for (int i = i0; i < re; i += kCgBlock) {
                    const RowSpan rs = row_span(a.slice_ptr, i);
                    const float ri = rg[i];
                    const float wi = spmv32_gather(a, rs, rg, ri);
                    wv[i - o] = wi;
                    g = fmaf(ri, ri, g);
                    d = fmaf(wi, ri, d);
                    ep = fmaf(a.v[i], ri, ep);
                }
            }
            double v3[3] = {(double)g, (double)d, (double)ep};
            if (!(ok = cg_grid_sum<3>(v3, CGCG_PART, a.bar, gen, a.spin, buf, tot))) break;
            if (threadIdx.x == 0) {
                const double gam = tot[0], del = tot[1], eps = tot[2];
                if (!isfinite(gam) || !isfinite(del)) {
                    sc.refresh = 2;
                } else if (gam <= sc.rel2 || gam <= sc.pred2 || it >= a.maxit) {
                    // refresh; sc.rho keeps r^.r^ of the previous iteration so
                    // that beta can be formed with the refreshed residual
                    sc.refresh = 1;
                } else {
                    const double beta = gam / sc.rho;
                    const double c = sc.deflate ? eps * sc.inv_mu : 0.0;
                    const double den = del - beta * gam / sc.alpha - eps * c;
                    if (!(den > 0.0) || !isfinite(den)) {
                        sc.refresh = 2;
                    } else {
                        sc.beta = beta;
                        sc.c = c;
                        sc.alpha = gam / den;
                        sc.rho = gam;
                    }
                }
            }
            __syncthreads();
            if (sc.refresh) break;
        }
        if (!ok) break;
        // fold the FP32 correction into the FP64 solution
        for (int i = i0; i < re; i += kCgBlock) a.x[i] += a.s64[i] * (double)el[i - o];
        if (threadIdx.x == 0 && sc.refresh == 2) sc.restart = 1;
        __syncthreads();
        if (!(ok = grid_sync(a.bar, gen, a.spin))) break;
    }
#undef CGCG_PART
    if (ok && sc.phase == 4)
        for (int i = i0; i < re; i += kCgBlock) a.x[i] = 0.0;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        const int ph = sc.phase;
        a.stats->iters = it;
        a.stats->status = !ok ? FV_E_TIMEOUT
                        : ph == 3 ? FV_E_DIVERGED : ph == 2 ? FV_E_NOT_CONVERGED : FV_OK;
        const bool zero = ph == 4;
        a.stats->res0 = zero ? 0.0 : sc.nr0 / sc.nb;
        a.stats->res = zero ? 0.0 : sc.nr / sc.nb;
        a.stats->outer = outer;
    }
}

// ------------------------------------------------------------ BiCGStab --

struct BicgArgs {
    int N, ncomp;
    const int32_t *slice_ptr, *col;
    const double *val, *diag, *b, *src, *gradp, *V;
    double *x, *dinv;
    double *r, *rh, *p, *v, *y, *s, *z, *t;   // [ncomp][N]
    double *partA, *partB;
    GridBar *bar;
    long long spin;
    double tol, reltol;
    int maxit;
    DevSolveStats *stats;
};

// A vec on row i for the components flagged in act: the row's coefficients
// and columns are read once for all components; each component's sum runs
// diagonal first, then the row's entries in slot order
template <int NC>
__device__ __forceinline__ void spmv_row_nc(const BicgArgs &a, int i, double d, const double *vec,
                                            const bool (&act)[NC], double (&out)[NC])
{
    const RowSpan rs = row_span(a.slice_ptr, i);
    const size_t NN = (size_t)a.N;
#pragma unroll
    for (int c = 0; c < NC; ++c) out[c] = act[c] ? d * vec[c * NN + i] : 0.0;
    for (int k = 0; k < rs.K; ++k) {
        const int e = rs.e0 + 32 * k;
        const double v = a.val[e];
        const size_t j = (size_t)a.col[e];
#pragma unroll
        for (int c = 0; c < NC; ++c)
            if (act[c]) out[c] += v * __ldcg(vec + c * NN + j);
    }
}

// Scalar state of a BiCGStab solve with NC right-hand sides, in shared memory
// and updated by thread 0 after each grid sum (as CgScalars); each pass copies
// the scalars it needs into registers.
template <int NC>
struct BicgScalars {
    double rho[NC], rho_old[NC], alpha[NC], omega[NC], beta[NC];
    double thr[NC], nb[NC], nr0[NC], nr[NC];
    int active[NC], iters[NC], status[NC];
    int n_active;
};

// NC components (1, or 3 for a momentum system) share the matrix.
template <int NC>
__global__ void __launch_bounds__(kBlock, 2) k_bicgstab(BicgArgs a)
{
    constexpr int nc = NC;
    const int N = a.N;
    const size_t NN = (size_t)N;
    const int stride = gridDim.x * kBlock;
    const int i0 = blockIdx.x * kBlock + threadIdx.x;
    unsigned gen = 0;
    bool ok = true;
    __shared__ BicgScalars<NC> sc;

    // S: r = b - A x, rh = r, norms per component
    double v6[6] = {0, 0, 0, 0, 0, 0};   // ||b_c||^2, ||r_c||^2
    bool act[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) act[c] = true;
    for (int i = i0; i < N; i += stride) {
        const double d = a.diag[i];
        a.dinv[i] = 1.0 / d;
        double ax[NC];
        spmv_row_nc<NC>(a, i, d, a.x, act, ax);
#pragma unroll
        for (int c = 0; c < nc; ++c) {
            const double bi = a.b ? a.b[c * NN + i] : a.src[c * NN + i] - a.V[i] * a.gradp[c * NN + i];
            const double ri = bi - ax[c];
            a.r[c * NN + i] = ri;
            a.rh[c * NN + i] = ri;
            v6[2 * c] += bi * bi;
            v6[2 * c + 1] += ri * ri;
        }
    }
    ok = grid_sum<6>(v6, a.partB, a.bar, gen, a.spin);
    if (threadIdx.x == 0) {
        sc.n_active = 0;
#pragma unroll
        for (int c = 0; c < nc; ++c) {
            sc.rho[c] = sc.rho_old[c] = sc.alpha[c] = sc.omega[c] = sc.beta[c] = 1.0;
            sc.thr[c] = sc.nb[c] = sc.nr0[c] = sc.nr[c] = 0.0;
            sc.active[c] = sc.iters[c] = sc.status[c] = 0;
            if (!ok) continue;
            const double nb = sqrt(v6[2 * c]);
            const double nr0 = sqrt(v6[2 * c + 1]);
            sc.thr[c] = fmax(a.tol * nb, a.reltol * nr0);
            sc.rho[c] = v6[2 * c + 1];
            sc.nb[c] = nb;
            if (nb != 0.0) {
                sc.nr0[c] = sc.nr[c] = nr0;
                if (nr0 > sc.thr[c]) { sc.active[c] = 1; ++sc.n_active; }
            }
        }
    }
    __syncthreads();
    if (ok) {
#pragma unroll
        for (int c = 0; c < nc; ++c)
            if (sc.nb[c] == 0.0)
                for (int i = i0; i < N; i += stride) a.x[c * NN + i] = 0.0;
    }
    int it = 0;
    while (ok && sc.n_active > 0) {
        ++it;
        // P1: p = r + beta (p - omega v); y = D^-1 p
        if (threadIdx.x == 0) {
#pragma unroll
            for (int c = 0; c < nc; ++c)
                sc.beta[c] = (sc.rho[c] / sc.rho_old[c]) * (sc.alpha[c] / sc.omega[c]);
        }
        __syncthreads();
        double beta[NC], omega[NC];
#pragma unroll
        for (int c = 0; c < nc; ++c) {
            act[c] = sc.active[c] != 0;
            beta[c] = sc.beta[c];
            omega[c] = sc.omega[c];
        }
        for (int i = i0; i < N; i += stride) {
            // every component's loads are issued before the first store
            const double di = a.dinv[i];
            double rr[NC], pp[NC], vv[NC];
#pragma unroll
            for (int c = 0; c < nc; ++c) {
                rr[c] = pp[c] = vv[c] = 0.0;
                if (!act[c]) continue;
                const size_t j = c * NN + i;
                rr[c] = a.r[j];
                if (it > 1) { pp[c] = a.p[j]; vv[c] = a.v[j]; }
            }
#pragma unroll
            for (int c = 0; c < nc; ++c) {
                if (!act[c]) continue;
                const size_t j = c * NN + i;
                const double pn = (it == 1) ? rr[c] : rr[c] + beta[c] * (pp[c] - omega[c] * vv[c]);
                a.p[j] = pn;
                a.y[j] = pn * di;
            }
        }
        if (!(ok = grid_sync(a.bar, gen, a.spin))) break;
        // P2: v = A y; rh.v
        double v3[3] = {0, 0, 0};
        for (int i = i0; i < N; i += stride) {
            const double d = a.diag[i];
            double rh[NC], ay[NC];
#pragma unroll
            for (int c = 0; c < nc; ++c) rh[c] = act[c] ? a.rh[c * NN + i] : 0.0;
            spmv_row_nc<NC>(a, i, d, a.y, act, ay);
#pragma unroll
            for (int c = 0; c < nc; ++c) {
                if (!act[c]) continue;
                a.v[c * NN + i] = ay[c];
                v3[c] += rh[c] * ay[c];
            }
        }
        if (!(ok = grid_sum<3>(v3, a.partA, a.bar, gen, a.spin))) break;
        if (threadIdx.x == 0) {
#pragma unroll
            for (int c = 0; c < nc; ++c) {
                if (!sc.active[c]) continue;
                if (v3[c] == 0.0 || !isfinite(v3[c])) {
                    sc.status[c] = FV_E_DIVERGED; sc.iters[c] = it; sc.active[c] = 0; --sc.n_active;
                } else {
                    sc.alpha[c] = sc.rho[c] / v3[c];
                }
            }
        }
        __syncthreads();
        double alpha[NC];
#pragma unroll
        for (int c = 0; c < nc; ++c) {
            act[c] = sc.active[c] != 0;
            alpha[c] = sc.alpha[c];
        }
        // P3: s = r - alpha v; z = D^-1 s
        for (int i = i0; i < N; i += stride) {
            const double di = a.dinv[i];
            double rr[NC], vv[NC];
#pragma unroll
            for (int c = 0; c < nc; ++c) {
                rr[c] = act[c] ? a.r[c * NN + i] : 0.0;
                vv[c] = act[c] ? a.v[c * NN + i] : 0.0;
            }
#pragma unroll
            for (int c = 0; c < nc; ++c) {
                if (!act[c]) continue;
                const size_t j = c * NN + i;
                const double si = rr[c] - alpha[c] * vv[c];
                a.s[j] = si;
                a.z[j] = si * di;
            }
        }
        if (!(ok = grid_sync(a.bar, gen, a.spin))) break;
        // P4: t = A z; t.s, t.t
        double w6[6] = {0, 0, 0, 0, 0, 0};
        for (int i = i0; i < N; i += stride) {
            const double d = a.diag[i];
            double ss[NC], az[NC];
#pragma unroll
            for (int c = 0; c < nc; ++c) ss[c] = act[c] ? a.s[c * NN + i] : 0.0;
            spmv_row_nc<NC>(a, i, d, a.z, act, az);
#pragma unroll
            for (int c = 0; c < nc; ++c) {
                if (!act[c]) continue;
                const double ti = az[c];
                a.t[c * NN + i] = ti;
                w6[2 * c] += ti * ss[c];
                w6[2 * c + 1] += ti * ti;
            }
        }
        if (!(ok = grid_sum<6>(w6, a.partB, a.bar, gen, a.spin))) break;
        if (threadIdx.x == 0) {
#pragma unroll
            for (int c = 0; c < nc; ++c)
                if (sc.active[c]) sc.omega[c] = w6[2 * c + 1] > 0.0 ? w6[2 * c] / w6[2 * c + 1] : 0.0;
        }
        __syncthreads();
#pragma unroll
        for (int c = 0; c < nc; ++c) omega[c] = sc.omega[c];
        // P5: x += alpha y + omega z; r = s - omega t; rh.r, r.r
        double u6[6] = {0, 0, 0, 0, 0, 0};
        for (int i = i0; i < N; i += stride) {
            double xn[NC], rn[NC], rh[NC];
#pragma unroll
            for (int c = 0; c < nc; ++c) {
                xn[c] = rn[c] = rh[c] = 0.0;
                if (!act[c]) continue;
                const size_t j = c * NN + i;
                xn[c] = a.x[j] + (alpha[c] * a.y[j] + omega[c] * a.z[j]);
                rn[c] = a.s[j] - omega[c] * a.t[j];
                rh[c] = a.rh[j];
            }
#pragma unroll
            for (int c = 0; c < nc; ++c) {
                if (!act[c]) continue;
                const size_t j = c * NN + i;
                a.x[j] = xn[c];
                a.r[j] = rn[c];
                u6[2 * c] += rh[c] * rn[c];
                u6[2 * c + 1] += rn[c] * rn[c];
            }
        }
        if (!(ok = grid_sum<6>(u6, a.partA, a.bar, gen, a.spin))) break;
        if (threadIdx.x == 0) {
#pragma unroll
            for (int c = 0; c < nc; ++c) {
                if (!sc.active[c]) continue;
                const double nr = sqrt(u6[2 * c + 1]);
                sc.nr[c] = nr;
                int stop = 0;
                if (!isfinite(nr)) { sc.status[c] = FV_E_DIVERGED; stop = 1; }
                else if (nr <= sc.thr[c]) { stop = 1; }
                else if (it >= a.maxit) { sc.status[c] = FV_E_NOT_CONVERGED; stop = 1; }
                else if (sc.omega[c] == 0.0) { sc.status[c] = FV_E_DIVERGED; stop = 1; }
                if (stop) { sc.iters[c] = it; sc.active[c] = 0; --sc.n_active; }
                sc.rho_old[c] = sc.rho[c];
                sc.rho[c] = u6[2 * c];
            }
        }
        __syncthreads();
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
#pragma unroll
        for (int c = 0; c < nc; ++c) {
            const double nb = sc.nb[c];
            a.stats[c].iters = sc.iters[c];
            a.stats[c].status = ok ? sc.status[c] : FV_E_TIMEOUT;
            a.stats[c].res0 = nb > 0.0 ? sc.nr0[c] / nb : 0.0;
            a.stats[c].res = nb > 0.0 ? sc.nr[c] / nb : 0.0;
            a.stats[c].outer = 1;
        }
    }
}

// ------------------------------------------------------------ launches --

static fv_status coop_launch(const void *fn, int G, int block, void **args, cudaStream_t s,
                             size_t smem = 0)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(G);
    cfg.blockDim = dim3(block);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    FV_CUDA(cudaLaunchKernelExC(&cfg, fn, args));
    return FV_OK;
}

static int grid_for(int rows, int block, int gmax)
{
    // about 4 rows per thread at least before another block is worth a
    // grid-wide barrier; never more blocks than can be co-resident
    int want = (rows + 4 * block - 1) / (4 * block);
    if (want < 1) want = 1;
    return want < gmax ? want : gmax;
}

// The CG launch: the resident form when the block's r^, q and y fit in the
// dynamic shared memory krylov_setup allowed, else the global form.
static fv_status launch_k_pcg(const fv_mesh *m, int G, CgArgs &a)
{
    void *args[] = {&a};
    const size_t res = (size_t)3 * sizeof(double) * cg_chunk(m->N, G);
    if (res <= (size_t)m->kw.cg_res_max)
        return coop_launch((const void *)k_pcg<true>, G, kCgBlock, args, m->stream, res);
    return coop_launch((const void *)k_pcg<false>, G, kCgBlock, args, m->stream);
}

// Dynamic shared memory a resident form may use: what a block can hold beyond
// the kernel's static shared memory, provided one block per SM stays resident
// with it.  0 (the global form) when the device cannot provide it; the
// resident form is an optimisation, so a failing query clears its error and
// leaves the global form in place instead of failing the mesh.
static int resident_room(const void *fn, bool allow)
{
    if (!allow) return 0;
    int dev = 0, optin = 0, per = 0;
    cudaFuncAttributes fa;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess ||
        cudaFuncGetAttributes(&fa, fn) != cudaSuccess) {
        (void)cudaGetLastError();
        return 0;
    }
    const int room = optin - (int)fa.sharedSizeBytes;
    if (room <= 0) return 0;
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, room) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, fn, kCgBlock, room) != cudaSuccess) {
        (void)cudaGetLastError();
        return 0;
    }
    return per >= 1 ? room : 0;
}

fv_status krylov_setup(fv_mesh *m)
{
    KrylovWork &w = m->kw;
    int per_sm = 0;
    FV_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_pcg<false>, kCgBlock, 0));
    FV_CHECK(per_sm >= 1, FV_E_CUDA, "CG kernel cannot be resident");
    // the resident CG forms may take what a block can hold beyond its static
    // shared memory, if one block per SM stays co-resident;
    // FVGB_CG_RESIDENT=0 keeps the global forms (tests compare the two)
    {
        const char *env = std::getenv("FVGB_CG_RESIDENT");
        const bool allow = !(env && std::atoi(env) == 0);
        w.cg_res_max = resident_room((const void *)k_pcg<true>, allow);
        w.mix_res_max = resident_room((const void *)k_pcg_mixed<true>, allow);
        w.cgcg_res_max = resident_room((const void *)k_pcg_mixed_cgcg<true>, allow);
        // order of the mixed-precision inner iterations: by default the
        // Chronopoulos-Gear order where its row vectors fit in shared
        // memory (synchronisation-bound there: 2 instead of 3 per
        // iteration), the textbook order otherwise (bandwidth-bound there,
        // and it moves fewer bytes); FVGB_MIXED_CG=classic or cgcg forces one
        const char *form = std::getenv("FVGB_MIXED_CG");
        w.mixed_form = !form ? 2 : std::strcmp(form, "classic") == 0 ? 0
                     : std::strcmp(form, "cgcg") == 0 ? 1 : 2;
    }
    FV_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_pcg_mixed_cgcg<false>, kCgBlock, 0));
    FV_CHECK(per_sm >= 1, FV_E_CUDA, "mixed CG kernel (Chronopoulos-Gear order) cannot be resident");
    FV_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_pcg_mixed<false>, kCgBlock, 0));
    FV_CHECK(per_sm >= 1, FV_E_CUDA, "mixed CG kernel cannot be resident");
    w.Gcg = m->sm_count;
    int per_sm2 = 0;
    FV_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm2, k_bicgstab<3>, kBlock, 0));
    FV_CHECK(per_sm2 >= 1, FV_E_CUDA, "BiCGStab kernel cannot be resident");
    w.block = kBlock;
    w.G = m->sm_count * (per_sm2 < 2 ? per_sm2 : 2);
    const size_t N = m->N;
    DeviceArena &ar = m->arena;
    fv_status st;
    if ((st = ar.alloc_n(&w.val, (size_t)m->nnz)) != FV_OK) return st;
    if ((st = ar.alloc_n(&w.val2, (size_t)m->nnz)) != FV_OK) return st;
    if ((st = ar.alloc_n(&w.dinv, N)) != FV_OK) return st;
    if ((st = ar.alloc_n(&w.r, N)) != FV_OK) return st;
    if ((st = ar.alloc_n(&w.p, N)) != FV_OK) return st;
    if ((st = ar.alloc_n(&w.q, N)) != FV_OK) return st;
    if ((st = ar.alloc_n(&w.y, N)) != FV_OK) return st;
    for (int k = 0; k < 8; ++k)
        if ((st = ar.alloc_n(&w.bv[k], 3 * N)) != FV_OK) return st;
    const int gp = w.G > w.Gcg ? w.G : w.Gcg;
    if ((st = ar.alloc_n(&w.partials, (size_t)2 * gp * kParts)) != FV_OK) return st;
    if ((st = ar.alloc_n(&w.bar, 1)) != FV_OK) return st;
    if ((st = ar.alloc_n(&w.stats, 4)) != FV_OK) return st;
    FV_CUDA(cudaMemsetAsync(w.bar, 0, sizeof(GridBar), m->stream));
    return FV_OK;
}

fv_status launch_pcg(const fv_mesh *m, const CgProblem &pb)
{
    const KrylovWork &w = m->kw;
    CgArgs a;
    a.N = m->N;
    a.slice_ptr = m->slice_ptr;
    a.col = m->col;
    a.val = pb.val;
    a.diag = pb.diag;
    a.b = pb.b;
    a.x = pb.x;
    a.s = w.dinv;
    a.r = w.r;
    a.p = w.p;
    a.q = w.q;
    a.y = w.y;
    const int gp = w.G > w.Gcg ? w.G : w.Gcg;
    a.partA = w.partials;
    a.partB = w.partials + (size_t)gp * kParts;
    a.bar = w.bar;
    a.spin = g_spin_limit;
    a.tol = pb.tol;
    a.reltol = pb.reltol;
    a.maxit = pb.maxit;
    a.stats = pb.stats;
    FV_CUDA(cudaMemsetAsync(w.bar, 0, sizeof(GridBar), m->stream));
    return launch_k_pcg(m, grid_for(m->N, kCgBlock, w.Gcg), a);
}

fv_status launch_pcg_mixed(const fv_mesh *m, const MixedProblem &pb)
{
    fv_mesh *mm = const_cast<fv_mesh *>(m);
    KrylovWork &w = mm->kw;
    if (!w.val32) {
        // FP32 work space, allocated once per mesh on first use
        DeviceArena &ar = mm->arena;
        fv_status st;
        if ((st = ar.alloc_n(&w.val32, (size_t)m->nnz)) != FV_OK) return st;
        for (int k = 0; k < 6; ++k)
            if ((st = ar.alloc_n(&w.f32[k], (size_t)m->N)) != FV_OK) return st;
    }
    const int G = grid_for(m->N, kCgBlock, w.Gcg);
    const int gp = w.G > w.Gcg ? w.G : w.Gcg;
    const bool cgcg_fits = (size_t)4 * sizeof(float) * cg_chunk(m->N, G) <= (size_t)w.cgcg_res_max;
    if (w.mixed_form == 1 || (w.mixed_form == 2 && cgcg_fits)) {
        if (!w.f32p[0]) {
            DeviceArena &ar = mm->arena;
            fv_status st;
            for (int k = 0; k < 2; ++k)
                if ((st = ar.alloc_n(&w.f32p[k], (size_t)m->N)) != FV_OK) return st;
        }
        CgcgArgs a;
        a.N = m->N;
        a.slice_ptr = m->slice_ptr;
        a.col = m->col;
        a.val = pb.val;
        a.val32 = w.val32;
        a.diag = pb.diag;
        a.b = pb.b;
        a.x = pb.x;
        a.s64 = w.dinv;
        a.r64 = w.r;
        a.a1 = w.y;
        a.r = w.f32[0];
        a.p = w.f32[1];
        a.e = w.f32[3];
        a.wd = w.f32[4];
        a.v = w.f32[5];
        a.sv = w.f32p[0];
        a.w = w.f32p[1];
        a.partA = w.partials;
        a.partB = w.partials + (size_t)gp * kParts;
        a.bar = w.bar;
        a.spin = g_spin_limit;
        a.tol = pb.tol;
        a.reltol = pb.reltol;
        a.maxit = pb.maxit;
        a.stats = pb.stats;
        FV_CUDA(cudaMemsetAsync(w.bar, 0, sizeof(GridBar), m->stream));
        void *args[] = {&a};
        const size_t res = (size_t)4 * sizeof(float) * cg_chunk(m->N, G);
        if (res <= (size_t)w.cgcg_res_max)
            return coop_launch((const void *)k_pcg_mixed_cgcg<true>, G, kCgBlock, args, m->stream, res);
        return coop_launch((const void *)k_pcg_mixed_cgcg<false>, G, kCgBlock, args, m->stream);
    }
    MixArgs a;
    a.N = m->N;
    a.slice_ptr = m->slice_ptr;
    a.col = m->col;
    a.val = pb.val;
    a.val32 = w.val32;
    a.diag = pb.diag;
    a.b = pb.b;
    a.x = pb.x;
    a.s = w.dinv;
    a.r64 = w.r;
    a.a1 = w.y;
    a.r = w.f32[0];
    a.p = w.f32[1];
    a.q = w.f32[2];
    a.e = w.f32[3];
    a.w = w.f32[4];
    a.v = w.f32[5];
    a.partA = w.partials;
    a.partB = w.partials + (size_t)gp * kParts;
    a.bar = w.bar;
    a.spin = g_spin_limit;
    a.tol = pb.tol;
    a.reltol = pb.reltol;
    a.maxit = pb.maxit;
    a.stats = pb.stats;
    FV_CUDA(cudaMemsetAsync(w.bar, 0, sizeof(GridBar), m->stream));
    void *args[] = {&a};
    const size_t res = (size_t)5 * sizeof(float) * cg_chunk(m->N, G);
    if (res <= (size_t)w.mix_res_max)
        return coop_launch((const void *)k_pcg_mixed<true>, G, kCgBlock, args, m->stream, res);
    return coop_launch((const void *)k_pcg_mixed<false>, G, kCgBlock, args, m->stream);
}

// Same CG launch with caller-supplied work vectors (the allocation-free
// entry point passes slices of its static scratch array).
fv_status launch_pcg_scratch(const fv_mesh *m, const CgProblem &pb, const CgScratch &ws)
{
    CgArgs a;
    a.N = m->N;
    a.slice_ptr = m->slice_ptr;
    a.col = m->col;
    a.val = pb.val;
    a.diag = pb.diag;
    a.b = pb.b;
    a.x = pb.x;
    a.s = ws.s;
    a.r = ws.r;
    a.p = ws.p;
    a.q = ws.q;
    a.y = ws.y;
    a.partA = ws.partials;
    a.partB = ws.partials + (size_t)ws.max_blocks * kParts;
    a.bar = ws.bar;
    a.spin = g_spin_limit;
    a.tol = pb.tol;
    a.reltol = pb.reltol;
    a.maxit = pb.maxit;
    a.stats = pb.stats;
    const int G = grid_for(m->N, kCgBlock, m->kw.Gcg);
    FV_CHECK(G <= ws.max_blocks, FV_E_INVALID, "scratch holds partial sums for %d blocks, %d needed",
             ws.max_blocks, G);
    FV_CUDA(cudaMemsetAsync(ws.bar, 0, sizeof(GridBar), m->stream));
    return launch_k_pcg(m, G, a);
}

fv_status launch_bicgstab(const fv_mesh *m, const BicgProblem &pb)
{
    const KrylovWork &w = m->kw;
    BicgArgs a;
    a.N = m->N;
    a.ncomp = pb.ncomp;
    a.slice_ptr = m->slice_ptr;
    a.col = m->col;
    a.val = pb.val;
    a.diag = pb.diag;
    a.b = pb.b;
    a.src = pb.src;
    a.gradp = pb.gradp;
    a.V = m->V;
    a.x = pb.x;
    a.dinv = w.dinv;
    a.r = w.bv[0];
    a.rh = w.bv[1];
    a.p = w.bv[2];
    a.v = w.bv[3];
    a.y = w.bv[4];
    a.s = w.bv[5];
    a.z = w.bv[6];
    a.t = w.bv[7];
    const int gp = w.G > w.Gcg ? w.G : w.Gcg;
    a.partA = w.partials;
    a.partB = w.partials + (size_t)gp * kParts;
    a.bar = w.bar;
    a.spin = g_spin_limit;
    a.tol = pb.tol;
    a.reltol = pb.reltol;
    a.maxit = pb.maxit;
    a.stats = pb.stats;
    FV_CUDA(cudaMemsetAsync(w.bar, 0, sizeof(GridBar), m->stream));
    void *args[] = {&a};
    FV_CHECK(pb.ncomp == 1 || pb.ncomp == 3, FV_E_INVALID, "BiCGStab takes 1 or 3 components, got %d",
             pb.ncomp);
    const void *fn = pb.ncomp == 3 ? (const void *)k_bicgstab<3> : (const void *)k_bicgstab<1>;
    return coop_launch(fn, grid_for(m->N, kBlock, w.G), kBlock, args, m->stream);
}

}  // namespace fvgb

extern "C" fv_status fv_set_barrier_spin_limit(int64_t limit)
{
    FV_CHECK(limit >= 0, FV_E_INVALID, "negative spin limit");
    fvgb::g_spin_limit = limit > 0 ? limit : (1LL << 25);
    return FV_OK;
}
