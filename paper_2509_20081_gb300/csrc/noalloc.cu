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

#include "dbt_internal.cuh"

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
// memory, so the device address is looked up once per device (with that
// device current) and cached.
constexpr int kMaxDevices = 64;
void *g_scratch_addr[kMaxDevices] = {};
std::mutex g_scratch_mutex;

cudaError_t scratch_address(void **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_scratch_mutex);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return cudaSuccess;
}

}  // namespace

// The first call on a device also looks up the scratch array's device
// address (cudaGetSymbolAddress); make that first call before capturing a
// stream into a CUDA graph.
extern "C" dbt_status dbt_integrate_scan_noalloc(const dbt_grid *g, const dbt_kernels *k,
                                                 const float *d_xyz, int64_t n,
                                                 const double pose[12], dbt_scan_stats *h_stats,
                                                 void *stream) {
    void *scratch = nullptr;
    const cudaError_t e = scratch_address(&scratch);
    if (e != cudaSuccess) return dbt::report_cuda_error(e, "cudaGetSymbolAddress(no-allocation scratch)");
    return dbt::integrate_on_scratch(g, k, d_xyz, n, pose, scratch, kScratchBytes, kMaxPoints,
                                     h_stats, (cudaStream_t)stream);
}
