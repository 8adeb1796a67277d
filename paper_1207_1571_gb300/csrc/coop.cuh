// coop.cuh -- the grid barrier and the deterministic reductions shared by
// the persistent cooperative solvers (krylov.cu, amg.cu).
//
// The barrier spins a bounded number of times on an arrival counter and
// otherwise records FV_E_TIMEOUT; reductions add per-thread partials in a
// fixed order inside a block and then the per-block partials in a fixed
// order, so every block obtains the same bits.
#pragma once

#include "fvgb_internal.h"

namespace fvgb {

constexpr int kParts = 8;       // doubles per block per partial record

__device__ __forceinline__ unsigned ld_acquire(const unsigned *p)
{
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void red_add_release(unsigned *p, unsigned v)
{
    asm volatile("red.release.gpu.global.add.u32 [%0], %1;" :: "l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ int ld_relaxed(const int *p)
{
    int v;
    asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Grid barrier.  Each block arrives with a release reduction on one
// counter, which only grows within a launch (the host zeroes it before
// each), and polls the counter with acquire loads until it holds the
// gridDim.x * (g + 1) arrivals of generation g.  Every arrival is an atomic
// read-modify-write, so the value a poller reads continues the release
// sequence of each earlier arrival and its acquire load orders all blocks'
// writes before the phase (made visible to the arriving thread by the
// block barrier) before its later reads; the block barrier then extends
// that to the block.  No block can arrive for generation g + 1 before every
// block has arrived for g, so counts past the target are harmless.  (A flat
// poll of the counter takes 1.2 us per barrier over 152 blocks, against 1.7
// us when the last arrival publishes a separate generation word.)  A waiter
// gives up after `limit` polls and records FV_E_TIMEOUT; waiters also leave
// when another block has recorded an error.  Returns false (for every
// thread of the block) in both cases.
__device__ inline bool grid_sync(GridBar *bar, unsigned &gen, long long limit)
{
    __shared__ int s_ok;
    __syncthreads();
    if (gridDim.x == 1) return true;
    if (threadIdx.x == 0) {
        int ok = 1;
        const unsigned target = (gen + 1) * gridDim.x;
        red_add_release(&bar->count, 1u);
        long long spins = 0;
        while ((int)(ld_acquire(&bar->count) - target) < 0) {
            ++spins;
            if (spins > limit) {
                atomicExch(&bar->err, FV_E_TIMEOUT);
                ok = 0;
                break;
            }
            if ((spins & 63) == 0 && ld_relaxed(&bar->err) != 0) {
                ok = 0;
                break;
            }
            if (spins > 256) __nanosleep(32);
        }
        s_ok = ok;
    }
    ++gen;
    __syncthreads();
    return s_ok != 0;
}

// Reductions keep FP64 work low: GB300 runs FP64 at about 2 FMA per clock
// per SM, and an FP64 warp instruction holds its sub-partition's FP64 pipe
// for ~64 cycles whatever its number of active lanes, so the cost of a sum
// is its count of FP64 warp instructions and its depth.  Threads drop their
// partial sums into shared memory, four warps add them in shallow trees, and
// one warp adds the four results and shuffles; after the grid barrier one
// warp per value adds the per-block partials.  Every order is fixed.

constexpr int kCgBlock = 1024;
constexpr int kRedWarps = 4;        // one reducing warp per SM sub-partition

__device__ __forceinline__ double warp_sum(double x)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    return x;
}

// Block sum of NV values over BLOCK threads.  Threads store their partials
// in shared memory; lane l of warp w (w = 0..3, one per SM sub-partition, so
// their FP64 work runs in parallel) adds the BLOCK/128 values
// w*BLOCK/4 + l + 32 j in a pairwise tree; warp 0 adds the four warps'
// values of each lane, (w0 + w1) + (w2 + w3), and sums its lanes with
// shuffles.  For BLOCK = 1024 that is 7 + 8 FP64 instructions of depth 3 + 7,
// against 13 + 4 of depth 17 for sequential lane sums and a single-thread
// final sum.  On return tot[k] (shared) holds the sums; only thread 0 is
// guaranteed to have seen them before the trailing __syncthreads of the
// caller.
template <int NV, int BLOCK = kCgBlock>
__device__ __forceinline__ void cg_block_sum(const double (&v)[NV], double (*buf)[BLOCK],
                                             double *tot)
{
    static_assert(kRedWarps == 4 && BLOCK % (32 * kRedWarps) == 0, "block size");
    constexpr int per = BLOCK / (32 * kRedWarps);      // values per lane
    __shared__ double lanes[NV][kRedWarps][32];
#pragma unroll
    for (int k = 0; k < NV; ++k) buf[k][threadIdx.x] = v[k];
    __syncthreads();
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (w < kRedWarps) {
#pragma unroll
        for (int k = 0; k < NV; ++k) {
            double t[per];
#pragma unroll
            for (int j = 0; j < per; ++j) t[j] = buf[k][w * (BLOCK / kRedWarps) + lane + 32 * j];
#pragma unroll
            for (int s = 1; s < per; s <<= 1)
#pragma unroll
                for (int j = 0; j + s < per; j += 2 * s) t[j] += t[j + s];
            lanes[k][w][lane] = t[0];
        }
    }
    __syncthreads();
    if (w == 0) {
#pragma unroll
        for (int k = 0; k < NV; ++k) {
            double x = (lanes[k][0][lane] + lanes[k][1][lane]) + (lanes[k][2][lane] + lanes[k][3][lane]);
            x = warp_sum(x);
            if (lane == 0) tot[k] = x;
        }
    }
}

// Grid sum of NV values; on return thread 0 of every block holds the same
// bits in tot[] (shared).  Returns false (all threads) if the barrier failed.
template <int NV, int BLOCK = kCgBlock>
__device__ inline bool cg_grid_sum(const double (&v)[NV], double *part, GridBar *bar, unsigned &gen,
                                   long long limit, double (*buf)[BLOCK], double *tot)
{
    cg_block_sum<NV, BLOCK>(v, buf, tot);
    if (gridDim.x == 1) return true;
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < NV; ++k) part[blockIdx.x * kParts + k] = tot[k];
    }
    if (!grid_sync(bar, gen, limit)) return false;
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (w < NV) {
        // warp k adds quantity k over the blocks: lane l the partials of
        // blocks l, l + 32, ... in that order (loads issued first), then the
        // lanes by shuffles
        const int G = gridDim.x;
        double x;
        if (G <= 32 * 8) {
            double t[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const int b = lane + 32 * j;
                t[j] = b < G ? __ldcg(part + b * kParts + w) : 0.0;
            }
            const int nslot = (G + 31) >> 5;
            x = t[0];
#pragma unroll
            for (int j = 1; j < 8; ++j)
                if (j < nslot) x += t[j];
        } else {
            x = 0.0;
            for (int j = lane; j < G; j += 32) x += __ldcg(part + j * kParts + w);
        }
        x = warp_sum(x);
        if (lane == 0) tot[w] = x;
    }
    __syncthreads();
    return true;
}

}  // namespace fvgb
