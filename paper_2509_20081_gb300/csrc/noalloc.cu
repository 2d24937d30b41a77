// dbt_integrate_scan_noalloc: scan integration for callers that cannot
// allocate device memory.
//
// Some callers are not allowed to call cudaMalloc once they are running: a
// real-time mapping loop that forbids allocation after start-up (allocation
// can block and its latency is unbounded), a plugin whose host framework owns
// every device allocation, or code that must stay within a memory budget
// fixed at start-up.  dbt_integrate_scan needs a caller-allocated workspace;
// this entry point instead uses a fixed scratch array compiled into the
// library, so a call allocates nothing.  The caller still passes the grid,
// the kernel tables and the returns.
//
// The array lives in device global memory of every GPU on which the library
// is loaded, for as long as the process runs, whether or not this entry point
// is ever called.  Every call shares it and it keeps the previous call's
// contents, so each call clears the parts that must start at zero, and calls
// whose work overlaps on the GPU (for example on two streams) race on it.
#include <mutex>

#include <cudaTypedefs.h>

#include "dbt_internal.cuh"
#include "scratch_cache.h"

// Limits of the fixed scratch: scans of up to 65,536 returns, and grids whose
// integration layout fits in 22 MiB: every grid of up to 524,288 bricks of
// 32 x 8 x 8 voxels (e.g. 1600 x 1600 x 320 voxels) at kernel sizes up to
// 17, and up to ~500,000 bricks at K = 19 or 21, whose returns touch up to
// 32 bricks each (~2.7 MB of per-return regions, no host staging, 4 B per
// pair slot, 24 B per brick).  Larger layouts are refused with DBT_EINVAL.
static constexpr long long kMaxPoints = 65536;
static constexpr size_t kScratchBytes = size_t(22) << 20;

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

namespace {

// In host code g_scratch names a host-side shadow of the symbol, not device
// memory.  Its device address belongs to the context the call runs in, so it
// is looked up (cudaGetSymbolAddress) the first time a context is seen and
// remembered under the context's unique id; a later context on the same
// device (after cudaDeviceReset, or a driver context of the caller's own)
// gets its own lookup.  When the driver cannot report context ids, every
// call looks the address up.
ContextAddressCache<64> g_cache;
std::mutex g_scratch_mutex;
PFN_cuCtxGetId_v12000 g_ctx_id = nullptr;
bool g_ctx_id_tried = false;

bool current_context_id(unsigned long long *id) {
    return g_ctx_id && g_ctx_id(nullptr, id) == CUDA_SUCCESS;
}

cudaError_t scratch_address(void **out) {
    std::lock_guard<std::mutex> lock(g_scratch_mutex);
    if (!g_ctx_id_tried) {
        g_ctx_id_tried = true;
        void *fn = nullptr;
        cudaDriverEntryPointQueryResult q{};
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &fn, 12000, cudaEnableDefault, &q) ==
                cudaSuccess && q == cudaDriverEntryPointSuccess)
            g_ctx_id = reinterpret_cast<PFN_cuCtxGetId_v12000>(fn);
        else
            (void)cudaGetLastError();
    }
    unsigned long long id = 0;
    if (current_context_id(&id)) {
        if (void *p = g_cache.find(id)) {
            *out = p;
            return cudaSuccess;
        }
    }
    // first call in this context (the lookup also makes the runtime's
    // context current when none was)
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess) return e;
    if (current_context_id(&id)) g_cache.put(id, p);
    *out = p;
    return cudaSuccess;
}

}  // namespace

// Host-only check of the no-allocation limits for a grid of nx x ny x nz
// voxels (rows padded to a multiple of 32), kernel size K and n returns;
// makes no CUDA call.
extern "C" dbt_status dbt_noalloc_check(int32_t nx, int32_t ny, int32_t nz, int32_t kernel_size,
                                        int64_t n) {
    if (nx < 1 || ny < 1 || nz < 1 || nx > 0x7FFFFFE0)
        return dbt::report_einval("grid dims must be >= 1 (nx <= 2^31 - 32)");
    const int32_t pitch = (int32_t)(((long long)nx + 31) / 32 * 32);
    return dbt::scratch_fits(pitch, ny, nz, kernel_size, n, kScratchBytes, kMaxPoints);
}

// The first call in a context also looks up the scratch array's device
// address (cudaGetSymbolAddress); make that first call before capturing a
// stream into a CUDA graph.
extern "C" dbt_status dbt_integrate_scan_noalloc(const dbt_grid *g, const dbt_kernels *k,
                                                 const float *d_xyz, int64_t n,
                                                 const double pose[12], dbt_scan_stats *h_stats,
                                                 void *stream) {
    // inputs the scratch cannot hold are refused before any CUDA call
    dbt_status st = dbt::scratch_fits_grid(g, k, n, kScratchBytes, kMaxPoints);
    if (st != DBT_OK) return st;
    void *scratch = nullptr;
    const cudaError_t e = scratch_address(&scratch);
    if (e != cudaSuccess) return dbt::report_cuda_error(e, "cudaGetSymbolAddress(no-allocation scratch)");
    return dbt::integrate_on_scratch(g, k, d_xyz, n, pose, scratch, kScratchBytes, kMaxPoints,
                                     h_stats, (cudaStream_t)stream);
}
