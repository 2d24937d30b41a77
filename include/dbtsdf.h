/*
 * dbtsdf.h -- C ABI of the GB300 DB-TSDF scan-integration library.
 *
 * DB-TSDF (arXiv 2509.20081) stores a dense voxel grid whose voxels hold a
 * 32-bit distance mask, a sign flag and a hit counter (Sec. III-A).  Each
 * LiDAR return selects a precomputed directional kernel by its direction
 * bin (Sec. III-B, Eq. 2) and updates the K^3 neighbourhood of its contact
 * voxel: masks are ANDed with the kernel's distance masks (Eqs. 3-4), and
 * the voxels of the hemispherical shadow get a saturating hit count and,
 * on crossing the threshold, the occupied sign (Eqs. 5-6).
 *
 * Conventions
 *  - Every function returns a dbt_status; nothing throws across the ABI.
 *    Argument errors are reported synchronously (DBT_EINVAL) with a message
 *    in dbt_last_error().  Work is enqueued asynchronously on the given
 *    CUDA stream (a cudaStream_t passed as void*; NULL = legacy default
 *    stream).  Device-side errors are latched in the workspace and reported
 *    by dbt_sync() / dbt_get_scan_stats().
 *  - The caller owns every device buffer (grid arrays, point buffers, the
 *    workspace scratch) and every stream.  The library owns only the kernel
 *    tables made by dbt_kernels_build() and small host-side handles.
 *  - Device pointers are marked d_, host pointers h_.  Pointers must stay
 *    valid until the enqueued work has finished.
 *  - Grid layout: three Structure-of-Arrays planes, each [nz][ny][pitch_x]
 *    with x fastest; voxel (x, y, z) is element (z * ny + y) * pitch_x + x.
 *    pitch_x = nx rounded up to a multiple of 32 (dbt_grid_layout); mask
 *    rows are 128-byte aligned when the array base is 256-byte aligned,
 *    which every base pointer must be.  Padding voxels (x >= nx) are
 *    initialised and never changed by integration.
 *  - Thread safety: calls on different grids/workspaces may run from
 *    different host threads; one workspace must not be used by two scans
 *    at the same time.
 */
#ifndef DBTSDF_H
#define DBTSDF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    DBT_OK = 0,
    DBT_EINVAL = 1,    /* bad argument; nothing was enqueued */
    DBT_ENOMEM = 2,    /* host/device allocation failed, or a buffer is too small */
    DBT_ECUDA = 3,     /* a CUDA runtime call failed (message in dbt_last_error) */
    DBT_ETIMEOUT = 4,  /* a bounded device-side wait gave up */
    DBT_ESTATE = 5     /* the device latched an error in the workspace */
} dbt_status;

typedef enum {
    DBT_BINS_OCTA = 0, /* n x n octahedral cells (bins_a = bins_b = n) */
    DBT_BINS_AZEL = 1  /* Eq. 2: bins_a = B_az azimuth x bins_b = B_el elevation */
} dbt_bin_scheme;

/* Kernel and update parameters (Sec. III-B, III-C).
 *  kernel_size   K, odd, 1..21 (the paper uses 21); neighbourhood [-R, R]^3,
 *                R = (K - 1) / 2.
 *  scheme        dbt_bin_scheme.
 *  bins_a/b      octa: n and n, 1 <= n <= 64; azel: B_az, B_el in 1..256
 *                (the paper uses 40 x 40).
 *  shadow_radius r_s in voxels, 0 <= r_s (the shadow is clipped to the
 *                kernel cube).
 *  hit_threshold T, 1 <= T <= hit_max (Eq. 6).
 *  hit_max       H_max, 1 <= H_max <= 65535 (Eq. 5).
 *  dedup_first   1: only the first return (lowest index) per contact voxel
 *                and scan is integrated (Sec. IV-B); 0: every return.
 *  shadow_cos    shape of the shadow (Sec. III-B): offset o of the ball
 *                |o| <= r_s is in the shadow of bin b when
 *                o . v_b >= shadow_cos * sqrt(|o|^2 |v_b|^2), v_b the bin's
 *                direction.  0 gives the paper's hemisphere; c in (0, 1] a
 *                cone of half-angle acos(c) around the ray (the conical
 *                model the paper compares against).  Finite, in [0, 1]. */
typedef struct {
    int32_t kernel_size;
    int32_t scheme;
    int32_t bins_a;
    int32_t bins_b;
    double shadow_radius;
    int32_t hit_threshold;
    int32_t hit_max;
    int32_t dedup_first;
    int32_t reserved;  /* must be 0 */
    double shadow_cos;
} dbt_params;

/* A dense grid.  mask/sign/hits are device arrays of pitch_x * ny * nz
 * elements each (uint32 / uint8 / uint16), 256-byte aligned.  res > 0 is
 * the voxel edge in metres; origin is the map-frame corner of voxel 0. */
typedef struct {
    uint32_t *mask;
    uint8_t *sign;
    uint16_t *hits;
    int32_t nx, ny, nz;
    int32_t pitch_x;
    double res;
    double origin[3];
} dbt_grid;

/* Opaque directional kernel tables (Eq. 3 distance masks, per-bin shadow
 * sets, Eq. 2 bin edges), built on the host and uploaded once; shareable by
 * any number of grids and streams. */
typedef struct dbt_kernels dbt_kernels;

/* Counters of the last completed scan of a workspace. */
typedef struct {
    int64_t n_input;    /* returns handed in */
    int64_t n_valid;    /* finite and not at the sensor origin */
    int64_t n_inside;   /* K^3 neighbourhood inside the grid (Sec. III-C) */
    int64_t n_kept;     /* integrated after the first-return rule */
    int64_t n_pairs;    /* (return, brick) work items */
    int64_t n_bricks;   /* bricks touched */
    uint32_t error;     /* device error bits, 0 = none */
    uint32_t reserved;
} dbt_scan_stats;

/* Eq. 1 sizing for the build's layout: pitch_x and bytes of each plane.
 * Any output pointer may be NULL.  EINVAL for non-positive or too large
 * dimensions (pitch_x * ny * nz must fit in 2^40 voxels). */
dbt_status dbt_grid_layout(int32_t nx, int32_t ny, int32_t nz, int32_t *pitch_x,
                           size_t *mask_bytes, size_t *sign_bytes, size_t *hits_bytes);

/* Sec. III-A initial state on every voxel (padding included): mask all ones,
 * sign free (1), hits 0.  Asynchronous on stream. */
dbt_status dbt_grid_init(const dbt_grid *g, void *stream);

/* Builds the kernel tables for p on the host and uploads them (synchronous;
 * allocates device memory owned by *out).  EINVAL on a bad parameter. */
dbt_status dbt_kernels_build(const dbt_params *p, dbt_kernels **out);

/* Frees the tables.  The caller must make sure no enqueued work uses them. */
dbt_status dbt_kernels_destroy(dbt_kernels *k);

/* Host copies of the tables, for checking them against an independent
 * build.  h_mask: K^3 uint32 Eq. 3 masks, [oz][oy][ox] with o + R as the
 * index.  h_shadow: bins * K^3 bytes, 1 where offset o is in the shadow of
 * bin b (Sec. III-B).  Either pointer may be NULL. */
dbt_status dbt_kernels_export(const dbt_kernels *k, uint32_t *h_mask, uint8_t *h_shadow);

/* The same tables built on the host only (no GPU needed), in the layout of
 * dbt_kernels_export: h_mask K^3 uint32, h_shadow bins * K^3 bytes. */
dbt_status dbt_tables_host(const dbt_params *p, uint32_t *h_mask, uint8_t *h_shadow);

/* Bin id of each direction (Eq. 2 or octahedral), computed on the device by
 * the same routine the integration uses: d_dirs n x 3 float64 map-frame
 * directions, d_bins n int32 outputs (-1 for a zero direction).  Async. */
dbt_status dbt_bin_directions(const dbt_kernels *k, const double *d_dirs, int64_t n,
                              int32_t *d_bins, void *stream);

/* The first steps of Sec. III-C for every return of a scan, without
 * integrating (the same device routine the integration starts with):
 * d_out[4 i .. 4 i + 3] = (x, y, z, bin), the contact voxel and direction bin
 * of return i, or (-1, 0, 0, 0) when the return is not valid (non-finite,
 * at the sensor origin) or its K^3 neighbourhood leaves the grid (boundary
 * discard).  The first-return rule is not applied and the grid is not read
 * or written.  d_xyz: device float32 n x 3 (sensor frame); pose as for
 * dbt_integrate_scan; d_out: device int32 n x 4, caller-owned.  Enqueued on
 * `stream`; DBT_EINVAL on bad arguments (nothing enqueued). */
dbt_status dbt_scan_contacts(const dbt_grid *g, const dbt_kernels *k, const float *d_xyz,
                             int64_t n, const double pose[12], int32_t *d_out, void *stream);

/* Handle over a caller-owned device scratch buffer used by integration: the
 * first-return hash table, per-return records, brick counters and the
 * (return, brick) work lists.  The handle is host memory; the library never
 * allocates device memory for it.  One workspace serves one grid geometry
 * and one scan at a time. */
typedef struct dbt_workspace dbt_workspace;

/* Bytes of device scratch a workspace needs for grid g, tables k and scans
 * of up to max_points returns (max_points >= 1).  The brick counters and
 * pair lists are sized for the shallowest brick depth (4), so the workspace
 * can be tuned to any depth (dbt_tuning). */
dbt_status dbt_workspace_size(const dbt_grid *g, const dbt_kernels *k, int64_t max_points,
                              size_t *bytes);

/* Wraps d_buf (256-byte aligned, >= dbt_workspace_size bytes, owned by the
 * caller) and zero-fills it asynchronously on stream. */
dbt_status dbt_workspace_create(const dbt_grid *g, const dbt_kernels *k, int64_t max_points,
                                void *d_buf, size_t bytes, void *stream, dbt_workspace **out);

/* Zero-fills the scratch again (after a device error or an aborted scan). */
dbt_status dbt_workspace_reset(dbt_workspace *ws, void *stream);

/* Frees the handle (not the caller's device buffer). */
dbt_status dbt_workspace_destroy(dbt_workspace *ws);

/* Integrates one scan (Sec. III-C).  d_xyz: n returns, float32 xyz
 * interleaved (12 bytes each, 4-byte aligned), in the sensor frame; NaN,
 * inf and origin returns are discarded.  pose: row-major 3x4 [R | t]
 * float64 (host memory, read before return), sensor frame -> map frame; R
 * must be a rotation (orthonormal to 1e-6, det > 0).  0 <= n <= the
 * workspace's max_points; g must have the geometry the workspace was made
 * for.  Asynchronous on stream; leaves the workspace ready for the next
 * scan. */
dbt_status dbt_integrate_scan(const dbt_grid *g, const dbt_kernels *k, dbt_workspace *ws,
                              const float *d_xyz, int64_t n, const double pose[12],
                              void *stream);

/* ---- Update pre-steps (Sec. III-C, Sec. IV-B) ---- */

/* Options of dbt_integrate_scan_ex.
 *  downsample  DS >= 1: sequential downsampling, only returns whose index is
 *              a multiple of DS are handed to the update (Sec. IV-B; the
 *              others count as not handed in: neither valid nor kept).
 *  n_poses     0: one pose for the scan (the pose argument).  1..256:
 *              motion compensation (Sec. III-C): return i is transformed
 *              with poses[m(i)], m(i) = ((i mod period) * n_poses) / period
 *              (integer division): the sweep's time runs with the index
 *              modulo period and is cut into n_poses equal slices.  For a
 *              beam-major spinning scan of W azimuths per beam, period = W;
 *              for returns stored in acquisition order, period = n.
 *  period      >= 1 when n_poses > 0.
 *  poses       host, n_poses x 12 (row-major 3x4 [R | t] each, checked like
 *              pose), read before the call returns (copied into the
 *              workspace on stream from pageable memory, so a call with
 *              n_poses > 0 cannot be captured into a CUDA graph). */
typedef struct {
    int32_t downsample;
    int32_t n_poses;
    int64_t period;
    const double *poses;
} dbt_scan_options;

/* dbt_integrate_scan with the options above (opt == NULL: the plain call;
 * pose may be NULL when opt->n_poses > 0).  Bit-identical to the plain
 * update of the downsampled returns, each under its slice's pose. */
dbt_status dbt_integrate_scan_ex(const dbt_grid *g, const dbt_kernels *k, dbt_workspace *ws,
                                 const float *d_xyz, int64_t n, const double pose[12],
                                 const dbt_scan_options *opt, void *stream);

typedef enum {
    DBT_MOTION_FULL = 0, /* R(tau) = R0 Exp(tau Log(R0^T R1)): constant angular velocity */
    DBT_MOTION_YAW = 1   /* R(tau) = Rz(tau dpsi) R0, dpsi = wrapped yaw(R1) - yaw(R0) */
} dbt_motion_mode;

/* Motion-compensation poses for a sweep from pose start to pose end (the
 * paper's "yaw-only or full SE(3)" compensation; its formula is not given,
 * these are this library's readings): out[12 m ..] = the pose at
 * tau_m = (m + 0.5) / n_poses, m < n_poses <= 256, rotation per mode and
 * translation t0 + tau (t1 - t0).  Host only. */
dbt_status dbt_pose_ramp(const double start[12], const double end[12], int32_t n_poses,
                         int32_t mode, double *out);

/* dbt_integrate_scan from host memory: copies the n returns at h_xyz into
 * one of the workspace's two staging buffers (on a copy stream the workspace
 * creates at its first call, so that the copy overlaps the previous scan's
 * kernels; pinned memory keeps it asynchronous), integrates them on
 * `stream` once the copy is done, and delivers the scan's counters to
 * *h_stats (8-byte aligned pinned host memory is written by the integrate
 * kernel itself; other host memory gets a copy on `stream`), which must stay
 * valid until the stream reaches that point.
 * h_xyz must stay unchanged until `stream` has passed this scan.
 * Asynchronous.  Workspaces of this call belong to one device. */
dbt_status dbt_integrate_scan_host(const dbt_grid *g, const dbt_kernels *k, dbt_workspace *ws,
                                   const float *h_xyz, int64_t n, const double pose[12],
                                   dbt_scan_stats *h_stats, void *stream);

/* Measurement hooks (not needed for integration).
 * dbt_workspace_set_timing: when the events are non-NULL, every later scan
 * on ws records ev_begin just before and ev_end just after its brick
 * integration kernel (cudaEvent_t passed as void*; NULL to stop).
 * dbt_scan_footprint: counts, for the scan (same arguments as
 * dbt_integrate_scan, grid left unchanged), the distinct voxels covered by
 * the K^3 neighbourhoods of its kept returns (h_counts[0] = U) and by their
 * shadow sets (h_counts[1] = U_s), i.e. the voxels whose state integration
 * must read and may write.  d_bits: caller scratch of at least
 * 2 * ceil(pitch_x * ny * nz / 32) * 4 + 16 bytes.  Synchronous. */
dbt_status dbt_workspace_set_timing(dbt_workspace *ws, void *ev_begin, void *ev_end);
dbt_status dbt_scan_footprint(const dbt_grid *g, const dbt_kernels *k, dbt_workspace *ws,
                              const float *d_xyz, int64_t n, const double pose[12], void *d_bits,
                              size_t bits_bytes, int64_t h_counts[2], void *stream);

/* Measurement hook: peak rates of the elementary updates the integration is
 * built from (the op-side ceiling of Eq. 7, T_update ~ N_p K^3 C_op),
 * measured alone by a micro-benchmark on the current device at the
 * integration's occupancy: *and_per_s = Eq. 4 voxel-ANDs per second as
 * byte-wise minima of packed 4-voxel code words in shared memory (the
 * faster of always / only-when-changed stores), *count_per_s = Eq. 5 counter
 * increments per second (16-bit counters in shared memory).  iters in
 * [16, 2^24] sets the loop length (2^14 takes a few ms).  Synchronous on
 * the default stream; allocates and frees 8 bytes of device memory. */
dbt_status dbt_op_rates(int32_t iters, double *and_per_s, double *count_per_s);

/* Batches: many scans of many grids (maps of any size) integrated by one
 * launch sequence.  The result on every grid equals integrating its scans
 * one by one with dbt_integrate_scan, in any order: a scan's effect depends
 * only on its kept returns (Eq. 4 is an AND; Eqs. 5-6 depend only on the
 * total count), and the first-return rule applies per scan.  Each brick
 * touched by several scans is staged once.  The grids are fixed when the
 * batch is created; each set of items names a grid by index.  dbt_batch_run
 * only enqueues kernels and memsets, so it can be captured in a CUDA graph
 * and replayed while the items are unchanged. */
typedef struct dbt_batch dbt_batch;

typedef struct {
    int32_t grid;           /* index into the batch's grids */
    int32_t reserved;       /* must be 0 */
    int64_t n;              /* returns */
    const float *d_xyz;     /* device, n x 3 float32, sensor frame */
    double pose[12];        /* row-major [R | t], sensor -> map */
} dbt_batch_item;

/* Bytes of device scratch for a batch over n_grids grids (<= 256), up to
 * max_points returns in total and max_items scans per run (sized, like a
 * workspace, for every brick depth). */
dbt_status dbt_batch_size(const dbt_grid *grids, int32_t n_grids, const dbt_kernels *k,
                          int64_t max_points, int32_t max_items, size_t *bytes);

/* Wraps caller-owned device scratch d_buf (256-byte aligned) for the given
 * grids (copied; their arrays must stay valid) and uploads the grid table
 * (synchronous on stream). */
dbt_status dbt_batch_create(const dbt_grid *grids, int32_t n_grids, const dbt_kernels *k,
                            int64_t max_points, int32_t max_items, void *d_buf, size_t bytes,
                            void *stream, dbt_batch **out);

/* Checks and uploads the scans of the next run (the copy first waits for
 * earlier work on stream).  Items of one grid may appear in any number. */
dbt_status dbt_batch_set_items(dbt_batch *b, const dbt_batch_item *items, int32_t n_items,
                               void *stream);

/* Enqueues the integration of the current items (asynchronous). */
dbt_status dbt_batch_run(dbt_batch *b, void *stream);

/* Synchronises stream; per-scan counters of the last run for the first n
 * items (n_pairs / n_bricks are 0 per scan) and the run's totals (either
 * pointer may be NULL).  DBT_ESTATE when the device latched an error. */
dbt_status dbt_batch_stats(const dbt_batch *b, dbt_scan_stats *per_item, int32_t n,
                           dbt_scan_stats *total, void *stream);

/* Frees the handle (not the caller's buffer). */
dbt_status dbt_batch_destroy(dbt_batch *b);

/* ---- Tuning and autotuning (no counterpart in the paper: launch choices of
 * this implementation; every setting gives bit-identical maps) ----
 *  heavy_pairs     bricks with more (return, brick) pairs than this are
 *                  integrated by a whole CTA, the others by one warp
 *                  (default 64; >= 0).
 *  integrate_ctas  CTAs of the persistent integrate kernel; 0 = every SM
 *                  filled to its occupancy limit (the default); at most 4x
 *                  that.
 *  brick_depth     z-extent of the 32 x 8 x brick_depth voxel bricks the
 *                  integration is split into: 4, 8 or 16 (16 only up to
 *                  kernel_size 17); 0 = 8, the default.  Workspaces and
 *                  batches are laid out for every depth; the getters report
 *                  the depth in use (never 0).  Shallow bricks give more,
 *                  smaller work items (fewer pairs per brick); deep ones
 *                  fewer pairs per return. */
typedef struct {
    int32_t heavy_pairs;
    int32_t integrate_ctas;
    int32_t brick_depth;
} dbt_tuning;

dbt_status dbt_workspace_set_tuning(dbt_workspace *ws, const dbt_kernels *k, const dbt_tuning *t);
dbt_status dbt_workspace_get_tuning(const dbt_workspace *ws, dbt_tuning *t);
dbt_status dbt_batch_set_tuning(dbt_batch *b, const dbt_tuning *t);
dbt_status dbt_batch_get_tuning(const dbt_batch *b, dbt_tuning *t);

/* Times candidate tunings over n_trials runs of the batch's current items
 * (one warm-up run each) with CUDA events on stream, in two stages: every
 * brick_depth (8, 4, and 16 where allowed) x heavy_pairs 16..256 on the
 * occupancy-maximum grid, then the winner on three, two and one CTAs per SM.
 * Keeps the fastest in *best and sets it on the batch.  The items are integrated (1 + n_trials) times
 * per candidate, so the batch's grids end in an unspecified state: run it
 * on scratch grids of the production shapes (fresh maps, or copies), then
 * apply *best with dbt_batch_set_tuning.  Synchronous. */
dbt_status dbt_batch_autotune(dbt_batch *b, int32_t n_trials, void *stream, dbt_tuning *best);

/* The same for single-scan integration: times dbt_integrate_scan of one scan
 * into g (a scratch grid, left in an unspecified state) and sets the
 * fastest tuning on ws. */
dbt_status dbt_workspace_autotune(const dbt_grid *g, const dbt_kernels *k, dbt_workspace *ws,
                                  const float *d_xyz, int64_t n, const double pose[12],
                                  int32_t n_trials, void *stream, dbt_tuning *best);

/* dbt_integrate_scan for callers that cannot allocate device memory (the
 * paper has no counterpart; this is a deployment convenience).  Some callers
 * may not call cudaMalloc while they run -- a real-time mapping loop that
 * forbids allocation after start-up, or a plugin whose host framework owns
 * every device allocation -- so they cannot provide a workspace.  This entry
 * point uses a fixed scratch array compiled into the library instead and
 * allocates nothing (host or device).  Limits: n <= 65,536 returns per scan,
 * and the grid's integration layout must fit in 22 MiB (true for every grid
 * of up to 524,288 bricks of 32 x 8 x 8 voxels at K <= 17, ~500,000 bricks
 * at K = 19 or 21); larger inputs are rejected
 * with DBT_EINVAL and a message.  The 22 MiB array occupies device memory on
 * every GPU that loads the library until the process exits.  All calls share
 * it: calls whose work overlaps on the GPU race, so issue them on one stream
 * (or otherwise serialise them).  The first call in a CUDA context looks up
 * the array's device address in that context (the address is remembered per
 * context, so a context created later, e.g. after cudaDeviceReset, gets its
 * own); make that first call before capturing a stream into a graph.
 * Other arguments as dbt_integrate_scan; *h_stats (may be NULL) receives the
 * scan's counters asynchronously, like dbt_integrate_scan_host. */
dbt_status dbt_integrate_scan_noalloc(const dbt_grid *g, const dbt_kernels *k, const float *d_xyz,
                                      int64_t n, const double pose[12], dbt_scan_stats *h_stats,
                                      void *stream);

/* Whether dbt_integrate_scan_noalloc can take a scan of n returns on a grid
 * of nx x ny x nz voxels (rows padded to a multiple of 32, as
 * dbt_grid_layout pads them) at kernel size kernel_size: DBT_OK, or
 * DBT_EINVAL with the reason in dbt_last_error().  The entry point applies
 * the same check (to the grid's own pitch) before any CUDA call.  Host only:
 * no CUDA call, no GPU needed.  The paper has no counterpart. */
dbt_status dbt_noalloc_check(int32_t nx, int32_t ny, int32_t nz, int32_t kernel_size, int64_t n);

/* Synchronises stream and copies the last scan's counters (may be NULL).
 * Returns DBT_ESTATE when the device latched an error. */
dbt_status dbt_get_scan_stats(const dbt_workspace *ws, dbt_scan_stats *out, void *stream);

/* Reads voxels: d_idx n x 3 int32 voxel coordinates (x, y, z); writes
 * d_mask / d_sign / d_hits (any may be NULL).  Coordinates outside the grid
 * give mask 0xFFFFFFFF, sign 1, hits 0.  Async. */
dbt_status dbt_read_voxels(const dbt_grid *g, const int32_t *d_idx, int64_t n, uint32_t *d_mask,
                           uint8_t *d_sign, uint16_t *d_hits, void *stream);

/* Signed distance readout (the paper gives no formula; this library's
 * reading): sdf = (sign ? +1 : -1) * popcount(mask) * res, in metres, for
 * voxel coordinates d_idx (n x 3 int32); outside voxels give +32 res. */
dbt_status dbt_read_distance(const dbt_grid *g, const int32_t *d_idx, int64_t n, float *d_sdf,
                             void *stream);

/* ---- Map export (Sec. III-C, Fig. 3: the map is exported as a mesh by
 * Marching Cubes at iso = 0) ----
 *
 * A box is int32 {x0, y0, z0, bx, by, bz}: the voxels [x0, x0+bx) x
 * [y0, y0+by) x [z0, z0+bz), inside the grid (EINVAL otherwise). */

/* Signed distance (the readout of dbt_read_distance) of every voxel of the
 * box into d_out[(z * by + y) * bx + x], float32, caller-owned.  Async. */
dbt_status dbt_sdf_field(const dbt_grid *g, const int32_t box[6], float *d_out, void *stream);

/* Bytes of device scratch dbt_mesh_extract needs for this box. */
dbt_status dbt_mesh_scratch_size(const dbt_grid *g, const int32_t box[6], size_t *bytes);

/* Marching Cubes over the cells of the box (the (bx-1)(by-1)(bz-1) cubes
 * between voxel centres, numbered L = (k (by-1) + j) (bx-1) + i).  The field
 * is the readout in binary32, f = (sign ? +1 : -1) * popcount(mask) * res
 * (res and iso rounded to float); a corner is inside when f < iso; the vertex
 * on a crossed edge from lower corner a to upper corner b is at
 * t = (iso - f_a) / (f_b - f_a), coordinate origin + res * ((index + 0.5) +
 * t) along the edge (binary32, in this order); vertices are in the map
 * frame.  Triangles are ordered by cell, then by the
 * configuration table (dbt_mesh_table); each is 9 floats (three xyz
 * vertices) whose right-hand normal points to sdf > iso, and the surface of
 * the box is closed except where it meets the box's faces.
 *   d_scratch   >= dbt_mesh_scratch_size bytes, 256-byte aligned.
 *   d_tri       room for max_tri triangles (9 floats each); may be NULL when
 *               max_tri == 0 (count only).
 *   d_cell      NULL, or room for max_tri int64 cell numbers L.
 *   h_ntri      (host) the box's total triangle count; when it exceeds
 *               max_tri only the first max_tri are written.
 * Blocks until the count is known (the triangles are written asynchronously
 * afterwards on stream). */
dbt_status dbt_mesh_extract(const dbt_grid *g, const int32_t box[6], double iso, void *d_scratch,
                            size_t scratch_bytes, float *d_tri, int64_t *d_cell, int64_t max_tri,
                            int64_t *h_ntri, void *stream);

/* The Marching Cubes configuration table: h_ntri[256] triangles per
 * configuration (bit q set = corner q inside, q = x | 2y | 4z) and
 * h_edges[256 * 15] their edge ids, 3 per triangle.  Edge 4 a + j runs along
 * axis a from corner lo to lo + 2^a, lo = (j&1)<<1 | (j>>1)<<2 (a = 0),
 * (j&1) | (j>>1)<<2 (a = 1), j (a = 2). */
dbt_status dbt_mesh_table(uint8_t *h_ntri, uint8_t *h_edges);

/* Predicted points for the quality metrics: the centroid of each of n_tri
 * triangles (9 floats each, as written by dbt_mesh_extract) into d_out (3
 * floats each), ((a + b) + c) / 3 in binary32.  Async. */
dbt_status dbt_mesh_centroids(const float *d_tri, int64_t n_tri, float *d_out, void *stream);

/* ---- Reconstruction quality (Sec. IV-B, "Mapping results") ----
 * Point sets are device float32 xyz arrays (12 bytes a point, 4-byte
 * aligned, at most 2^31 points). */

/* Bytes of scratch dbt_nn_distances needs for n_ref reference points. */
dbt_status dbt_nn_scratch_size(int64_t n_ref, size_t *bytes);

/* d_dist[i] = Euclidean distance from query i to its nearest reference
 * point, exact (uniform-grid index over the bounding box of both sets,
 * rings searched until no closer point can remain), evaluated in binary32;
 * +inf when n_ref == 0.  d_scratch 256-byte aligned.  Async. */
dbt_status dbt_nn_distances(const float *d_ref, int64_t n_ref, const float *d_query,
                            int64_t n_query, void *d_scratch, size_t bytes, float *d_dist,
                            void *stream);

typedef struct {
    double accuracy;      /* mean predicted -> reference distance (m) */
    double completeness;  /* mean reference -> predicted distance (m) */
    double chamfer_l1;    /* (accuracy + completeness) / 2 */
    double precision;     /* fraction of predicted points with distance < tolerance */
    double recall;        /* fraction of reference points with distance < tolerance */
    double fscore;        /* 2 P R / (P + R), 0 when P + R = 0 */
    int64_t n_pred, n_gt;
} dbt_quality;

dbt_status dbt_quality_scratch_size(int64_t n_pred, int64_t n_gt, size_t *bytes);

/* The paper's metrics of a predicted point set against reference points at
 * a tolerance (m, finite, >= 0): distances from dbt_nn_distances, sums in
 * binary64 in a fixed order (the same result on every run).  An empty set
 * gives 0 for its own mean and fraction.  Synchronous (the result is copied
 * to *h_out). */
dbt_status dbt_quality_metrics(const float *d_pred, int64_t n_pred, const float *d_gt,
                               int64_t n_gt, double tolerance, void *d_scratch, size_t bytes,
                               dbt_quality *h_out, void *stream);

/* Synchronises stream and reports a latched device error of the workspace
 * (ws may be NULL to only synchronise). */
dbt_status dbt_sync(void *stream, const dbt_workspace *ws);

/* Message of the last failing call on this host thread ("" if none). */
const char *dbt_last_error(void);

/* Library version, e.g. "dbtsdf 0.1.0 sm_103a". */
const char *dbt_version(void);

#ifdef __cplusplus
}
#endif

#endif /* DBTSDF_H */
