// noalloc.cu -- a pressure CG solve that allocates no device memory.
//
// fv_pcg_solve keeps its work vectors in memory that fv_mesh_create
// allocated.  Some callers cannot let the library allocate at solve time:
// applications whose device memory is all handed out by their own allocator
// or pool and which forbid other code from calling cudaMalloc / cudaFree
// behind it, and code that runs while a CUDA stream capture in global mode is
// active elsewhere in the process, where allocation calls are refused.  For
// them, fv_pcg_solve_noalloc runs the same CG kernel with its work vectors
// in one fixed array of device memory that this file declares statically:
// the array exists on every GPU that loads the library, for as long as the
// library stays loaded, and every call uses the same array.
#include <mutex>

#include "coop.cuh"
#include "fvgb_internal.h"

namespace fvgb {
namespace {

// Limits of the static scratch array.
constexpr int kNoAllocMaxCells = 1 << 17;        // 131072 cells
constexpr int kNoAllocMaxEntries = 1 << 20;      // 1048576 row-structure entries
constexpr int kNoAllocMaxBlocks = 1024;          // partial sums of up to 1024 blocks

constexpr size_t align256(size_t n) { return (n + 255) & ~size_t(255); }
constexpr size_t kOffBar = 0;
constexpr size_t kOffStats = align256(kOffBar + sizeof(GridBar));
constexpr size_t kOffParts = align256(kOffStats + sizeof(DevSolveStats));
// two partial-sum records of kParts doubles per block (launch_pcg_scratch
// places the second at max_blocks * kParts)
constexpr size_t kOffVec = align256(kOffParts + sizeof(double) * 2 * kNoAllocMaxBlocks * kParts);
constexpr size_t kVecBytes = align256(sizeof(double) * (size_t)kNoAllocMaxCells);
constexpr size_t kOffVal = kOffVec + 5 * kVecBytes;
constexpr size_t kScratchBytes = align256(kOffVal + sizeof(double) * (size_t)kNoAllocMaxEntries);

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

// device address of the array on each device, looked up once per device
std::mutex g_mu;
constexpr int kMaxDevices = 64;
unsigned char *g_addr[kMaxDevices] = {};

// The array's address on the mesh's device.  cudaGetSymbolAddress answers
// for the current device, so the current device must be the mesh's.
fv_status scratch_address(const fv_mesh *m, unsigned char **out)
{
    int dev = 0;
    FV_CUDA(cudaGetDevice(&dev));
    FV_CHECK(dev == m->device, FV_E_INVALID,
             "fv_pcg_solve_noalloc: current device %d is not the mesh's device %d", dev, m->device);
    FV_CHECK(dev >= 0 && dev < kMaxDevices, FV_E_UNSUPPORTED, "device %d out of range", dev);
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_addr[dev]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_status(e, "cudaGetSymbolAddress(scratch)");
        g_addr[dev] = static_cast<unsigned char *>(p);
    }
    *out = g_addr[dev];
    return FV_OK;
}

}  // namespace
}  // namespace fvgb

using namespace fvgb;

extern "C" fv_status fv_pcg_solve_noalloc(const fv_mesh *mc, const double *diag,
                                          const double *upper, const double *b, double *x,
                                          const fv_pcg_params *prm, fv_solve_stats *stats)
{
    FV_CHECK(mc && diag && b && x && prm, FV_E_INVALID, "NULL argument");
    FV_CHECK(mc->F == 0 || upper, FV_E_INVALID, "upper is NULL");
    FV_CHECK(prm->maxit >= 0 && prm->tol >= 0.0 && prm->reltol >= 0.0, FV_E_INVALID, "bad params");
    FV_CHECK(mc->N <= kNoAllocMaxCells, FV_E_INVALID,
             "fv_pcg_solve_noalloc handles at most %d cells (mesh has %d)", kNoAllocMaxCells, mc->N);
    FV_CHECK(mc->nnz <= kNoAllocMaxEntries, FV_E_INVALID,
             "fv_pcg_solve_noalloc handles at most %d row entries (mesh has %d)",
             kNoAllocMaxEntries, mc->nnz);
    unsigned char *base = nullptr;
    fv_status st = scratch_address(mc, &base);
    if (st != FV_OK) return st;
    CgScratch ws;
    ws.bar = reinterpret_cast<GridBar *>(base + kOffBar);
    ws.partials = reinterpret_cast<double *>(base + kOffParts);
    ws.max_blocks = kNoAllocMaxBlocks;
    ws.s = reinterpret_cast<double *>(base + kOffVec + 0 * kVecBytes);
    ws.r = reinterpret_cast<double *>(base + kOffVec + 1 * kVecBytes);
    ws.p = reinterpret_cast<double *>(base + kOffVec + 2 * kVecBytes);
    ws.q = reinterpret_cast<double *>(base + kOffVec + 3 * kVecBytes);
    ws.y = reinterpret_cast<double *>(base + kOffVec + 4 * kVecBytes);
    double *val = reinterpret_cast<double *>(base + kOffVal);
    DevSolveStats *dstats = reinterpret_cast<DevSolveStats *>(base + kOffStats);
    fv_mesh *m = const_cast<fv_mesh *>(mc);
    if ((st = launch_ldu_to_sell(m, upper, upper, val)) != FV_OK) return st;
    CgProblem cp{diag, val, b, x, prm->tol, prm->reltol, prm->maxit, dstats};
    if ((st = launch_pcg_scratch(m, cp, ws)) != FV_OK) return st;
    DevSolveStats h;
    FV_CUDA(cudaMemcpyAsync(&h, dstats, sizeof(h), cudaMemcpyDeviceToHost, m->stream));
    FV_CUDA(cudaStreamSynchronize(m->stream));
    if (stats) {
        stats->iters = h.iters;
        stats->status = h.status;
        stats->res0 = h.res0;
        stats->res = h.res;
        stats->outer = h.outer;
        stats->pad_ = 0;
    }
    return (fv_status)h.status;
}
