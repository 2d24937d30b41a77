// Internal declarations shared by the library's translation units (never by
// the oracle).  Device-side layouts of the kernel tables, the grid view, the
// pose and the integration workspace.
#pragma once

#include <algorithm>
#include <cuda_runtime.h>
#include <stdint.h>

#include "dbtsdf.h"

namespace dbt {

// Brick = CTA ownership unit of the integration: BX x BY x BZ voxels.  BX = 32
// makes one brick row a 128-byte mask line; chunks are 4 voxels (16 bytes).
// The depth BZ is a launch choice (4, 8 or 16; 16 only up to K = 17, where a
// contact's brick-relative z still fits the pair payload's 5 bits): the grid
// view carries its log2 (bzs), the integrate kernel is instantiated per depth.
constexpr int BX = 32, BY = 8;
constexpr int CHUNKS_PER_ROW = BX / 4;      // 8
constexpr int BZ_DEFAULT = 8;
constexpr int BZ_MIN = 4;                   // the deepest brick count a scratch layout must hold
constexpr int BZ_MAX = 16;
constexpr int BZ16_MAX_K = 17;
__host__ __device__ constexpr int bz_shift(int bz) { return bz == 4 ? 2 : bz == 16 ? 4 : 3; }

constexpr int MAX_K = 21;
constexpr int MAX_R = (MAX_K - 1) / 2;
constexpr int MAX_M2 = 3 * MAX_R * MAX_R + 1;   // r^2 = 0 .. 3 R^2
constexpr int MAX_EDGES = 256;

// Device error bits latched in the workspace header.
constexpr uint32_t ERR_HASH_FULL = 1u << 0;
constexpr uint32_t ERR_PAIRS_OVERFLOW = 1u << 1;
constexpr uint32_t ERR_TOUCHED_OVERFLOW = 1u << 2;
constexpr uint32_t ERR_BAD_PAYLOAD = 1u << 3;
constexpr uint32_t ERR_MASK_FORM = 1u << 4;      // a grid mask was not of the form 2^k - 1

// Bricks a return's K^3 neighbourhood can touch with bricks of depth bz: its
// x-extent K spans at most 1 + ceil((K - 1) / BX) bricks, likewise in y and z.
__host__ __device__ inline int max_pairs_per_return(int K, int bz) {
    return (1 + (K - 1 + BX - 1) / BX) * (1 + (K - 1 + BY - 1) / BY) * (1 + (K - 1 + bz - 1) / bz);
}

// Shadow offsets are packed as bytes (ox + OFF_BIAS) | (oy + OFF_BIAS) << 8 |
// (oz + OFF_BIAS) << 16 (|o| <= MAX_R, so every byte is in [22, 42]).
constexpr int OFF_BIAS = 32;
__host__ __device__ inline uint32_t pack_off(int ox, int oy, int oz) {
    return (uint32_t)(ox + OFF_BIAS) | ((uint32_t)(oy + OFF_BIAS) << 8) |
           ((uint32_t)(oz + OFF_BIAS) << 16);
}
__host__ __device__ inline int off_axis(uint32_t o, int axis) {
    return (int)((o >> (8 * axis)) & 255u) - OFF_BIAS;
}

struct DevParams {
    int K, R;
    int scheme;       // DBT_BINS_OCTA / DBT_BINS_AZEL
    int na, nb;       // bins_a, bins_b
    int nbins;
    int T, Hmax;
    int dedup;
    int n_m2;         // entries of the mask-by-r^2 table
    int sr;           // min(R, floor(r_s)): no shadow offset exceeds it on any axis
    int n_sh;         // shadow offsets over all bins
};

struct DevTables {
    const uint32_t *m2;        // Eq. 3 mask as a function of r^2 = |o|^2
    const uint32_t *sh_off;    // packed shadow offsets, grouped by bin
    const uint32_t *sh_start;  // nbins + 1 prefix offsets into sh_off
    const double *az_c;        // azimuth edge k: cos(theta_k), k = 0..B_az-1
    const double *az_s;        // sin(theta_k)
    const int *az_up;          // theta_k < pi
    const double *el_s;        // elevation edge k: sin(phi_k), k = 0..B_el-1
    const uint32_t *prow;      // kernel-row codes P[q * (2R + 4) + s], q = 0 .. 2 R^2
    // shadow sub-ranges (sw = 2 sr + 1): sh_y lists each bin's offsets
    // oy-major (the same per-bin ranges as sh_off, which is oz-major);
    // sh_zs[b * (sw + 1) + k] / sh_ys[...] = first entry of bin b with
    // oz (resp. oy) >= k - sr in sh_off (resp. sh_y), k = 0 .. sw
    const uint32_t *sh_y;
    const uint32_t *sh_zs;
    const uint32_t *sh_ys;
};

struct DevGrid {
    uint32_t *mask;
    uint8_t *sign;
    uint16_t *hits;
    int nx, ny, nz, pitch;
    int nbx, nby, nbz;          // bricks per axis
    int bzs;                    // log2 of the brick depth BZ
    double res;                 // voxel edge (the binary64 voxel floor divides by it)
    double inv_res;             // 1 / res, rounded once on the host (binary32 filter data only)
    double ox, oy, oz;          // origin
};

struct Pose {
    double r[9];                // row-major rotation
    double t[3];
    // binary32 filter data for one grid (pose_filter): with b = (t - origin)
    // * inv_res in binary64 and B = round(b), the voxel coordinate along
    // axis k is fa[3k..3k+2] . p + fb[k] + B[k] up to a bounded error
    float fa[9];                // fl32(r * inv_res)
    float fr[9];                // fl32(r)
    float fb[3];                // fl32(b - B)
    int fbi[3];                 // B
    float fe0[3];               // absolute error allowance of fb[k] and of the binary64 path
    int fast;                   // 0: every return takes the binary64 path
};

// Fills the filter fields of P for grid g (host).
void pose_filter(Pose &P, const DevGrid &g);

// One scan of a batch: its returns, the grid (index into the batch's grid
// table) and the pose.
struct ItemDev {
    const float *xyz;
    long long n;
    int grid;
    int pad;
    Pose pose;
};

// Per-scan counters of a batch.
struct ItemCounters {
    unsigned long long valid, inside, kept, pad;
};

// Device tables of a batch: grids with the first global brick of each
// (bricks of all grids are numbered in one space), scans with the first
// return of each (returns of all scans in one index space).
struct BatchDev {
    const DevGrid *grids;      // n_grids
    const uint32_t *bbase;     // n_grids + 1
    const ItemDev *items;      // n_items
    const long long *istart;   // n_items + 1
    ItemCounters *icnt;        // n_items
    int n_grids, n_items;
    int bzs;                   // log2 of the brick depth of every grid view
};
constexpr int MAX_BATCH_GRIDS = 256;   // grid index lives in 8 bits of a return record
constexpr int MAX_BATCH_ITEMS = 1 << 20;

// Counters of the last completed scan; same layout as dbt_scan_stats.
struct ScanStats {
    long long n_input, n_valid, n_inside, n_kept, n_pairs, n_bricks;
    uint32_t error, reserved;
};
static_assert(sizeof(ScanStats) == sizeof(dbt_scan_stats), "stats layout");

// Light bricks are queued in size classes, the largest claimed first (a
// large brick taken last would leave most warps idle while it finishes):
// class c < LIGHT_CLASSES - 1 holds the bricks with more than heavy / 2^(c+1)
// pairs, the last class the rest.
constexpr int LIGHT_CLASSES = 5;
__host__ __device__ inline int light_class(uint32_t len, uint32_t heavy) {
    int c = 0;
    for (uint32_t t = heavy >> 1; c < LIGHT_CLASSES - 1 && len <= t; t >>= 1) ++c;
    return c;
}

struct WsHeader {
    uint32_t err;               // latched error bits of the current scan
    uint32_t n_touched;         // bricks touched by the current scan
    uint32_t pool;              // (return, brick) pairs allocated
    uint32_t next_work;         // dynamic queue of light bricks (one warp each)
    uint32_t done_ctas;         // integrate warps finished
    uint32_t n_heavy;           // bricks with more than `heavy` pairs (one CTA each)
    uint32_t next_heavy;        // dynamic queue of heavy bricks
    uint32_t n_vheavy;          // of those, bricks with more than 4 x `heavy` (taken first)
    unsigned long long acc_valid, acc_inside, acc_kept;
    uint32_t n_cls[LIGHT_CLASSES];   // light bricks per size class
    uint32_t next_vheavy;       // dynamic queue of very heavy bricks (whole CTAs)
    uint32_t pad1[7 - LIGHT_CLASSES];
    ScanStats last;             // published by the last integrate CTA
};

// Device view of a workspace (all pointers into the caller's buffer).
struct WsDev {
    WsHeader *hdr;
    float *stage;               // max_points * 3 floats (host-input staging)
    int4 *prec;                 // per return: contact (x,y,z) and bin, or x < 0
    unsigned long long *hkey;   // first-return hash: key = linear voxel + 1
    uint32_t *hidx;             // ~(lowest return index), 0 = empty
    uint32_t hcap_alloc;        // allocated slots (power of two)
    uint32_t *bcnt;             // per brick: pair count / fill cursor (kept 0 between scans)
    uint32_t *boff;             // per brick: first pair of its segment
    // Brick queues, max_touched entries each, filled from both ends: heavy
    // bricks at the front of order and the very heavy ones (more than 4 x
    // heavy pairs, taken first) at its back; light class c at the front
    // (even c) or back (odd c) of lq[c / 2].
    uint32_t *order;
    uint32_t *lq[3];
    uint32_t max_touched;
    uint32_t *pairs;            // pair payloads grouped by brick
    unsigned long long pairs_cap;
    Pose *poses;                // motion compensation: MAX_SCAN_POSES per-slice poses
    uint32_t heavy;             // bricks with more pairs than this go to a whole CTA
    uint32_t nbricks;           // bricks of the grid(s): the range of bcnt / boff
    // Host memory the device can write (pinned, mapped) that also receives
    // the scan's counters when they are published, or null.
    ScanStats *stats_out = nullptr;
};

__device__ __forceinline__ uint32_t *light_queue_slot(const WsDev &ws, int c, uint32_t q) {
    uint32_t *a = ws.lq[c >> 1];
    return a + ((c & 1) ? ws.max_touched - 1 - q : q);
}
constexpr uint32_t VHEAVY_FACTOR = 4;
static_assert(LIGHT_CLASSES == 5, "light_queue_slot places five classes");

// Update pre-steps of dbt_integrate_scan_ex: sequential downsampling (every
// ds-th return) and motion compensation (return i uses ws.poses[m(i)],
// m(i) = ((i mod period) * n_poses) / period).
struct ScanEx {
    int ds;
    int n_poses;
    long long period;
};
constexpr int MAX_SCAN_POSES = 256;

// Default of WsDev::heavy: bricks with more (return, brick) pairs than this
// are integrated by a whole CTA, the others by a single warp (tunable per
// workspace or batch; any value gives the same result).
constexpr uint32_t HEAVY_PAIRS = 64;

// Return record prec.w: bin in bits 0-15, batch grid index in bits 16-23,
// PREC_DUP when the first-return rule drops the return.
constexpr int PREC_DUP = 1 << 30;

// Programmatic dependent launch.  The kernels of a scan are launched with
// launch_pdl: the next kernel's CTAs may be scheduled while the previous
// kernel on the stream drains, which hides the launch gap.  pdl_wait()
// (griddepcontrol.wait) holds a thread until every prerequisite grid has
// completed and its writes are visible; a kernel launched without the
// attribute passes it at once.  Each of these kernels waits before it reads
// or writes global memory that any other kernel (or the caller) writes.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
// Lets the next kernel launch once every CTA of this grid has called it (or
// exited).
__device__ __forceinline__ void pdl_launch_dependents() {
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

template <typename... KArgs, typename... Args>
inline void launch_pdl(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                       Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    (void)cudaLaunchKernelEx(&cfg, kern, args...);   // errors surface through cudaGetLastError
}

// Launch helpers implemented in the .cu files.
void launch_voxelize(const DevGrid &g, const DevParams &p, const DevTables &t, const Pose &pose,
                     const float *xyz, int n, const WsDev &ws, uint32_t hcap, cudaStream_t s,
                     const ScanEx *ex = nullptr);

void launch_contacts(const DevGrid &g, const DevParams &p, const DevTables &t, const Pose &pose,
                     const float *xyz, long long n, int4 *out, cudaStream_t s);
void launch_alloc(const DevGrid &g, const DevParams &p, long long n, const WsDev &ws, uint32_t hcap,
                  cudaStream_t s);
void launch_alloc_batch(const BatchDev &bd, const DevParams &p, long long n, const WsDev &ws,
                        uint32_t hcap, cudaStream_t s);
void launch_fill(const DevGrid &g, const DevParams &p, int n, const WsDev &ws, uint32_t hcap,
                 cudaStream_t s);
void launch_integrate(const DevGrid &g, const DevParams &p, const DevTables &t, long long n_input,
                      const WsDev &ws, int grid_ctas, cudaStream_t s);
// Batched forms: every scan of bd at once (one brick pass over all grids).
void launch_voxelize_batch(const BatchDev &bd, const DevParams &p, const DevTables &t,
                           long long n, const WsDev &ws, uint32_t hcap, cudaStream_t s);

void launch_fill_batch(const BatchDev &bd, const DevParams &p, long long n, const WsDev &ws,
                       uint32_t hcap, cudaStream_t s);
void launch_integrate_batch(const BatchDev &bd, const DevParams &p, const DevTables &t,
                            long long n_input, const WsDev &ws, int grid_ctas, cudaStream_t s);
int integrate_grid_ctas(const DevParams &p, int bz);
int device_sm_count();
void launch_footprint(const DevGrid &g, const DevParams &p, const DevTables &t, int n,
                      const WsDev &ws, uint32_t hcap, uint32_t *bits_u, uint32_t *bits_s,
                      unsigned long long *counts, cudaStream_t s);
void launch_bin_dirs(const DevParams &p, const DevTables &t, const double *dirs, int n, int *bins,
                     cudaStream_t s);
void launch_read_voxels(const DevGrid &g, const int *idx, long long n, uint32_t *mask,
                        uint8_t *sign, uint16_t *hits, cudaStream_t s);
void launch_read_distance(const DevGrid &g, double res, const int *idx, long long n, float *sdf,
                          cudaStream_t s);

// Map export (export.cu).  A box of voxels [x0, x0+bx) x ...; its cells are
// the cx x cy x cz = (bx-1)(by-1)(bz-1) cubes between voxel centres.
struct ExportBox {
    int x0, y0, z0, bx, by, bz;
    long long cx, cy, cz, ncell;
};
void launch_sdf_field(const DevGrid &g, double res, const ExportBox &b, float *out, cudaStream_t s);
size_t mc_scratch_bytes(const ExportBox &b);
void launch_mc_count(const DevGrid &g, const ExportBox &b, uint64_t lut0, uint64_t lut1,
                     void *scratch, cudaStream_t s);
void launch_mc_emit(const DevGrid &g, const ExportBox &b, double res, double iso, uint64_t lut0,
                    uint64_t lut1, void *scratch, float *tri, long long *cell, long long max_tri,
                    cudaStream_t s);
const unsigned long long *mc_total_ptr(void *scratch);
void launch_exclusive_scan(const uint32_t *cnt, long long n, unsigned long long *out,
                           unsigned long long *tile, unsigned long long *total, cudaStream_t s);

// Quality metrics (quality.cu).
size_t nn_scratch_bytes(long long n_ref);
void launch_nn_distances(const float *ref, long long n_ref, const float *q, long long n_q,
                         void *scratch, float *dist, cudaStream_t s);
size_t quality_partials_bytes();
void launch_quality_reduce(const float *d_pred, long long n_pred, const float *d_gt,
                           long long n_gt, float tol, void *partials, double *out6,
                           cudaStream_t s);
void launch_centroids(const float *tri, long long n, float *out, cudaStream_t s);
void mc_table_host(uint8_t *ntri, uint8_t *edges);

// Sets the thread's error message for a failed CUDA call; returns DBT_ECUDA.
dbt_status report_cuda_error(cudaError_t e, const char *what);

// Limits of a fixed scratch of `bytes` for scans of up to max_points
// returns: n returns on a grid of pitch_x x ny x nz voxels at kernel size K
// (DBT_EINVAL with a message when they do not fit); host only, no CUDA call.
dbt_status scratch_fits(int32_t pitch_x, int32_t ny, int32_t nz, int32_t K, int64_t n,
                        size_t bytes, long long max_points);
// The same for grid g and kernels k (also checks the grid's fields).
dbt_status scratch_fits_grid(const dbt_grid *g, const dbt_kernels *k, int64_t n, size_t bytes,
                             long long max_points);
// Sets the thread's error message; returns DBT_EINVAL.
dbt_status report_einval(const char *msg);

// One scan on a caller-provided scratch buffer (see noalloc.cu); defined in api.cu.
dbt_status integrate_on_scratch(const dbt_grid *g, const dbt_kernels *k, const float *d_xyz,
                                int64_t n, const double pose[12], void *scratch,
                                size_t scratch_bytes, long long max_points,
                                dbt_scan_stats *h_stats, cudaStream_t s);

}  // namespace dbt
