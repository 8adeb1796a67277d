// coop.cuh -- the grid barrier and the deterministic reductions shared by
// the persistent cooperative solvers (krylov.cu, amg.cu).
//
// The barrier spins a bounded number of times on a generation counter and
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

__device__ __forceinline__ unsigned atom_add_acq_rel(unsigned *p, unsigned v)
{
    unsigned old;
    asm volatile("atom.add.acq_rel.gpu.global.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
    return old;
}

__device__ __forceinline__ void st_release(unsigned *p, unsigned v)
{
    asm volatile("st.release.gpu.global.u32 [%0], %1;" :: "l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ int ld_relaxed(const int *p)
{
    int v;
    asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Grid barrier.  The block's writes are ordered before its arrival by the
// block barrier and the release half of the arrival's atomic; the arrival
// counter only grows within a launch (the host zeroes it before each), so
// the last of the gridDim.x arrivals of generation g reads
// (g + 1) * gridDim.x - 1 and publishes g + 1 with a release store, which
// the waiters' acquire loads (then the block barrier) order before their
// later reads.  A waiter gives up after `limit` polls and records
// FV_E_TIMEOUT; waiters also leave when another block has recorded an
// error.  Returns false (for every thread of the block) in both cases.
__device__ inline bool grid_sync(GridBar *bar, unsigned &gen, long long limit)
{
    __shared__ int s_ok;
    __syncthreads();
    if (gridDim.x == 1) return true;
    if (threadIdx.x == 0) {
        int ok = 1;
        const unsigned g = gen;
        const unsigned old = atom_add_acq_rel(&bar->count, 1u);
        if (old == (g + 1) * gridDim.x - 1) {
            st_release(&bar->gen, g + 1);
        } else {
            long long spins = 0;
            while (ld_acquire(&bar->gen) == g) {
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
        }
        s_ok = ok;
    }
    ++gen;
    __syncthreads();
    return s_ok != 0;
}

// Reductions keep FP64 work low (GB300 runs FP64 at about 2 FMA per clock
// per SM): threads drop their partial sums into shared memory and one warp
// adds them in a fixed order; after the grid barrier one warp adds the
// per-block partials, again in a fixed order.

constexpr int kCgBlock = 1024;
constexpr int kRedWarps = 4;        // one reducing warp per SM sub-partition

__device__ __forceinline__ double warp_sum(double x)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    return x;
}

// Block sum of NV values over BLOCK threads.  Threads store their partials in shared memory;
// warps 0..3 (one per SM sub-partition, so their FP64 work runs in
// parallel) each add a quarter of them, then thread 0 adds the four results.
// The order of every addition is fixed.  On return tot[k] (shared) holds the
// sums; only thread 0 is guaranteed to have seen them before the trailing
// __syncthreads of the caller.
template <int NV, int BLOCK = kCgBlock>
__device__ __forceinline__ void cg_block_sum(const double (&v)[NV], double (*buf)[BLOCK],
                                             double *tot)
{
    __shared__ double quarter[NV][kRedWarps];
#pragma unroll
    for (int k = 0; k < NV; ++k) buf[k][threadIdx.x] = v[k];
    __syncthreads();
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (w < kRedWarps) {
        constexpr int per = BLOCK / kRedWarps;         // values per warp
#pragma unroll
        for (int k = 0; k < NV; ++k) {
            double x = 0.0;
#pragma unroll
            for (int j = 0; j < per / 32; ++j) x += buf[k][w * per + lane + 32 * j];
            x = warp_sum(x);
            if (lane == 0) quarter[k][w] = x;
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < NV; ++k) {
            double x = 0.0;
#pragma unroll
            for (int q = 0; q < kRedWarps; ++q) x += quarter[k][q];
            tot[k] = x;
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
        // warp k adds quantity k over the blocks
        double x = 0.0;
        for (int j = lane; j < (int)gridDim.x; j += 32) x += __ldcg(part + j * kParts + w);
        x = warp_sum(x);
        if (lane == 0) tot[w] = x;
    }
    __syncthreads();
    return true;
}

}  // namespace fvgb
