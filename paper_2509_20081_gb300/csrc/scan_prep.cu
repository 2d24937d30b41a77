// Per-return stages of one scan (Sec. III-C), before the brick integration:
//   k_voxelize  map-frame transform, contact voxel, boundary discard,
//               direction bin, first-return hash insert, and the
//               (return, brick) pair counts of each distinct contact voxel
//   k_alloc     first-return resolve; one contiguous pair segment per
//               touched brick
//   k_fill      pair payloads into the segments; clears the hash table
// plus the direction-bin and voxel readout kernels.
//
// Float -> integer decisions are the binary64 evaluation of Sec. III-C's
// formulas as written, each operation an explicit round-to-nearest
// intrinsic so that nvcc cannot contract or reorder them:
//   d = R p, row r = (R_r0 * x + R_r1 * y) + R_r2 * z; w = d + t
//   c = floor((w - origin) / res), a true division
//   octahedral: u = d_x / s, v = d_y / s, s = (|x| + |y|) + |z|
//   Eq. 2: edge comparisons against host-built cos/sin tables.
// A binary32 filter with rigorous error bounds reaches the same decisions
// without binary64 for all but the returns near a boundary.
#include "dbt_internal.cuh"

namespace dbt {

// ------------------------------------------------------------------ bins
__device__ __forceinline__ double sgn1(double v) { return v < 0.0 ? -1.0 : 1.0; }

// Octahedral cell of d (the workloads' scheme): projection on |x|+|y|+|z|=1,
// lower half folded over the diagonals, [-1,1]^2 cut into n x n cells.
__device__ int bin_octa(double dx, double dy, double dz, int n) {
    double s = __dadd_rn(__dadd_rn(fabs(dx), fabs(dy)), fabs(dz));
    if (!(s > 0.0)) return 0;
    double u = __ddiv_rn(dx, s);
    double v = __ddiv_rn(dy, s);
    if (dz < 0.0) {
        // (1 - |v|) sgn(u): a multiplication by +-1 is an exact sign choice
        const double fu = __dsub_rn(1.0, fabs(v)), fv = __dsub_rn(1.0, fabs(u));
        u = sgn1(u) < 0.0 ? -fu : fu;
        v = sgn1(v) < 0.0 ? -fv : fv;
    }
    // floor and the clamp to [0, n - 1] in integers (the conversion rounds
    // toward -inf: the same integer as floor() on the binary64 value)
    const int i = __double2int_rd(__dmul_rn(__dmul_rn(__dadd_rn(u, 1.0), 0.5), (double)n));
    const int j = __double2int_rd(__dmul_rn(__dmul_rn(__dadd_rn(v, 1.0), 0.5), (double)n));
    return min(max(j, 0), n - 1) * n + min(max(i, 0), n - 1);
}

// Eq. 2 azimuth: number of edges theta_k (k >= 1) with theta >= theta_k.
// Within a half-turn the test is the sign of cos(theta_k) y - sin(theta_k) x;
// the predicate falls monotonically with k, so a binary search finds the
// count.
__device__ __forceinline__ bool az_ge(const DevTables &t, int k, double x, double y, bool upper) {
    bool eu = t.az_up[k] != 0;
    if (upper && !eu) return false;
    if (!upper && eu) return true;
    return __dsub_rn(__dmul_rn(t.az_c[k], y), __dmul_rn(t.az_s[k], x)) >= 0.0;
}

__device__ int bin_az(const DevTables &t, int B, double x, double y) {
    if (x == 0.0 && y == 0.0) return 0;          // atan2(0, 0) = 0
    bool upper = (y > 0.0) || (y == 0.0 && x >= 0.0);
    int lo = 0, hi = B - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (az_ge(t, mid, x, y, upper)) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// Eq. 2 elevation: number of edges k >= 1 with z/|d| >= sin(phi_k); the
// top bin is B_el - 1 (clamped zenith).
__device__ int bin_el(const DevTables &t, int B, double x, double y, double z) {
    double nrm = __dsqrt_rn(__dadd_rn(__dadd_rn(__dmul_rn(x, x), __dmul_rn(y, y)), __dmul_rn(z, z)));
    double s = __ddiv_rn(z, nrm);
    int lo = 0, hi = B - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (s >= t.el_s[mid]) lo = mid; else hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ int bin_of(const DevParams &p, const DevTables &t, double dx, double dy,
                                      double dz) {
    if (p.scheme == DBT_BINS_OCTA) return bin_octa(dx, dy, dz, p.na);
    return bin_el(t, p.nb, dx, dy, dz) * p.na + bin_az(t, p.na, dx, dy);
}

// ------------------------------------------------------------------ hash
__device__ __forceinline__ uint32_t hslot(unsigned long long key, uint32_t hcap) {
    return (uint32_t)((key * 0x9E3779B97F4A7C15ull) >> 32) & (hcap - 1);
}

// First-return rule (Sec. IV-B): the slot of a contact voxel keeps the
// bitwise complement of the lowest return index seen, via atomicMax.
// Returns true for the one insert that created the slot (the voxel's first
// insert in time, not necessarily its lowest index).
__device__ bool hash_insert(const WsDev &ws, uint32_t hcap, unsigned long long key, uint32_t i) {
    uint32_t s = hslot(key, hcap);
    for (uint32_t probe = 0; probe < hcap; ++probe) {
        unsigned long long prev = atomicCAS(&ws.hkey[s], 0ull, key);
        if (prev == 0ull || prev == key) {
            atomicMax(&ws.hidx[s], ~i);
            return prev == 0ull;
        }
        s = (s + 1) & (hcap - 1);
    }
    atomicOr(&ws.hdr->err, ERR_HASH_FULL);
    return false;
}

__device__ bool hash_is_first(const WsDev &ws, uint32_t hcap, unsigned long long key, uint32_t i) {
    uint32_t s = hslot(key, hcap);
    for (uint32_t probe = 0; probe < hcap; ++probe) {
        unsigned long long k = ws.hkey[s];
        if (k == key) return ws.hidx[s] == ~i;
        if (k == 0ull) break;
        s = (s + 1) & (hcap - 1);
    }
    atomicOr(&ws.hdr->err, ERR_HASH_FULL);
    return false;
}

__device__ __forceinline__ unsigned long long voxel_key(const DevGrid &g, int x, int y, int z) {
    return ((unsigned long long)z * (unsigned long long)g.ny + (unsigned long long)y) *
               (unsigned long long)g.pitch + (unsigned long long)x + 1ull;
}

// ------------------------------------------------------------------ filter
// The voxel and octahedral-cell decisions are floors of binary64 values.
// They are first taken from binary32 evaluations with a rigorous bound on
// their distance to the exact real value (a floating-point filter in the
// sense of Shewchuk's adaptive predicates): when the binary32 value lies
// farther than its bound from every integer, the binary64 value (within
// ~2^-50 relative of the same real value) has the same floor.  Otherwise,
// and for poses without filter data, the binary64 path decides.
//
// Allowance of a binary32 sum of three products and a constant taken by
// FMAs (3 roundings) with binary32-rounded coefficients (1 more): 4u (1 +
// 4u) < 2.4e-7 relative to the sum of the terms' magnitudes, u = 2^-24;
// 3.5e-7 leaves room for the rounding of the allowance itself.
constexpr float FILTER_REL = 3.5e-7f;
// Absolute allowance for products that fall into the binary32 subnormal
// range (each loses at most 2^-150).
constexpr float FILTER_ABS = 1e-37f;

// floor(v) when every real within e of v has the same floor; false when
// uncertain or NaN.  v - f and (f + 1) - v are exact or off by <= 2^-25,
// far below every allowance passed in.
__device__ __forceinline__ bool floor_certain(float v, float e, long long &q) {
    const float f = floorf(v);
    if (!(v - f > e && (f + 1.0f) - v > e)) return false;
    q = (long long)f;
    return true;
}

// bin_octa from binary32 directions d with absolute error bounds e; -1 when
// a decision is uncertain.  |s - s*| <= es; |d_x / s - d*_x / s*| <= (e_x +
// es) / s because |d*_x| <= s*; each later binary32 operation adds one
// rounding of a value of magnitude <= 2 (<= 1.2e-7) before the scaling by
// n / 2.
__device__ __forceinline__ int bin_octa_f32(const float d[3], const float e[3], int n) {
    const float ax = fabsf(d[0]), ay = fabsf(d[1]), az = fabsf(d[2]);
    const float s = (ax + ay) + az;
    const float es = (e[0] + e[1] + e[2]) * 1.001f + s * 2.5e-7f;
    if (!(s > 4.0f * es) || !(az > e[2])) return -1;        // fold decision uncertain
    float u = __fdiv_rn(d[0], s), v = __fdiv_rn(d[1], s);
    float eu = __fdiv_ru(e[0] + es, s) * 1.01f + 1.2e-7f;
    float ev = __fdiv_ru(e[1] + es, s) * 1.01f + 1.2e-7f;
    if (d[2] < 0.0f) {
        if (!(ax > e[0] && ay > e[1])) return -1;          // signs of u, v uncertain
        const float fu = 1.0f - fabsf(v), fv = 1.0f - fabsf(u);
        const float eu0 = eu;
        eu = ev + 1.2e-7f;
        ev = eu0 + 1.2e-7f;
        u = d[0] < 0.0f ? -fu : fu;
        v = d[1] < 0.0f ? -fv : fv;
    }
    const float h = 0.5f * (float)n;
    const float au = (u + 1.0f) * h, av = (v + 1.0f) * h;
    long long i, j;
    if (!floor_certain(au, (eu + 2.4e-7f) * h * 1.01f + fabsf(au) * 1.2e-7f + 1e-6f, i) ||
        !floor_certain(av, (ev + 2.4e-7f) * h * 1.01f + fabsf(av) * 1.2e-7f + 1e-6f, j))
        return -1;
    return (int)(min(max(j, 0ll), (long long)n - 1) * n + min(max(i, 0ll), (long long)n - 1));
}

// ------------------------------------------------------------------ counters
// Scan counters of one CTA.  Every warp of the grid adding its popcounts to
// one global address would serialise those atomics at L2 (thousands per
// launch); the warps add into shared memory instead and one thread per CTA
// adds the totals.  Batches also count per scan: a CTA's consecutive
// returns belong to a few consecutive scans, counted in a window of
// TALLY_ITEMS slots from the CTA's first scan (scans past it add directly).
constexpr int TALLY_ITEMS = 8;
constexpr int TALLY_FLAGS = 3;            // valid, inside, kept
struct CtaTally {
    uint32_t hdr[TALLY_FLAGS];
    uint32_t item[TALLY_ITEMS][TALLY_FLAGS];
    int first_item;
};

__device__ __forceinline__ void tally_init(CtaTally &s, int first_item) {
    if (threadIdx.x < TALLY_FLAGS) s.hdr[threadIdx.x] = 0u;
    if (threadIdx.x < TALLY_FLAGS * TALLY_ITEMS)
        s.item[threadIdx.x / TALLY_FLAGS][threadIdx.x % TALLY_FLAGS] = 0u;
    if (threadIdx.x == 0) s.first_item = first_item;
    __syncthreads();
}

// Warp popcounts of the three flags into the CTA's header tallies.
__device__ __forceinline__ void tally_warp(CtaTally &s, const bool f[TALLY_FLAGS]) {
#pragma unroll
    for (int k = 0; k < TALLY_FLAGS; ++k) {
        const unsigned b = __ballot_sync(0xffffffffu, f[k]);
        if ((threadIdx.x & 31) == 0 && b) atomicAdd(&s.hdr[k], (uint32_t)__popc(b));
    }
}

// After the CTA's last tally: its totals to the scan counters.
__device__ __forceinline__ void tally_flush(CtaTally &s, const WsDev &ws) {
    __syncthreads();
    if (threadIdx.x == 0) {
        if (s.hdr[0]) atomicAdd(&ws.hdr->acc_valid, (unsigned long long)s.hdr[0]);
        if (s.hdr[1]) atomicAdd(&ws.hdr->acc_inside, (unsigned long long)s.hdr[1]);
        if (s.hdr[2]) atomicAdd(&ws.hdr->acc_kept, (unsigned long long)s.hdr[2]);
    }
}

// ------------------------------------------------------------------ pairs
// Brick range of the K^3 neighbourhood of contact c along one axis.
struct BrickSpan {
    int x0, x1, y0, y1, z0, z1;
};
__device__ __forceinline__ BrickSpan brick_span(int cx, int cy, int cz, int R, int bzs) {
    BrickSpan s;
    s.x0 = (cx - R) / BX;  // contacts are >= R, so these are non-negative
    s.x1 = (cx + R) / BX;
    s.y0 = (cy - R) / BY;
    s.y1 = (cy + R) / BY;
    s.z0 = (cz - R) >> bzs;
    s.z1 = (cz + R) >> bzs;
    return s;
}

// The (up to 2 x 4 x 4) bricks of each lane's pair span; f(valid, brick,
// bx, by, bz) per brick.  AGG: enumerated in lock-step over the warp (steps
// past a lane's own span call f with valid = false) so that lanes naming one
// brick can add together.
template <bool AGG, typename F>
__device__ __forceinline__ void for_pair_bricks(bool has, const BrickSpan &s, const DevGrid &g,
                                                uint32_t b0, F f) {
    const int sx = s.x1 - s.x0 + 1, sy = s.y1 - s.y0 + 1, sz = s.z1 - s.z0 + 1;
    const int np = has ? sx * sy * sz : 0;
    const int nsteps = AGG ? __reduce_max_sync(0xffffffffu, np) : np;
    int ix = 0, iy = 0, iz = 0;
    for (int j = 0; j < nsteps; ++j) {
        const bool v = j < np;
        const uint32_t b = v ? b0 + ((uint32_t)(s.z0 + iz) * g.nby + (s.y0 + iy)) * g.nbx + (s.x0 + ix)
                             : 0u;
        f(v, b, s.x0 + ix, s.y0 + iy, s.z0 + iz);
        if (++ix == sx) {
            ix = 0;
            if (++iy == sy) {
                iy = 0;
                ++iz;
            }
        }
    }
}

// Pair counts per brick.  The counts are fire-and-forget atomics (nothing
// waits for their old value); k_alloc finds the touched bricks afterwards
// by scanning the counters.  AGG: lanes naming one brick add together.
template <bool AGG>
__device__ __forceinline__ void count_pairs(const WsDev &ws, const DevGrid &g, uint32_t b0,
                                            bool kept, const BrickSpan &s) {
    for_pair_bricks<AGG>(kept, s, g, b0, [&](bool v, uint32_t b, int, int, int) {
        if constexpr (AGG) {
            const unsigned peers = __match_any_sync(0xffffffffu, v ? b : 0xFFFFFFFFu);
            if (v && (threadIdx.x & 31) == __ffs(peers) - 1) atomicAdd(&ws.bcnt[b], (uint32_t)__popc(peers));
        } else {
            if (v) atomicAdd(&ws.bcnt[b], 1u);
        }
    });
}

// ------------------------------------------------------------------ K1
// Map-frame direction d = R p in binary64, each row (r0 x + r1 y) + r2 z
// with every product and sum rounded on its own (no fused multiply-add).
__device__ __forceinline__ void direction64(const Pose &pose, double px, double py, double pz,
                                            double d[3]) {
#pragma unroll
    for (int r = 0; r < 3; ++r)
        d[r] = __dadd_rn(__dadd_rn(__dmul_rn(pose.r[3 * r + 0], px), __dmul_rn(pose.r[3 * r + 1], py)),
                         __dmul_rn(pose.r[3 * r + 2], pz));
}

// Sec. III-C for one return: discard non-finite and origin returns, map-frame
// transform, contact voxel, boundary discard, bin.  Returns 0 (not valid),
// 1 (valid, outside) or 2 (inside, rec filled with contact and bin).
__device__ __forceinline__ int contact_of(const DevGrid &g, const DevParams &p, const DevTables &t,
                                          const Pose &pose, float fx, float fy, float fz,
                                          int4 &rec) {
    if (!(isfinite(fx) && isfinite(fy) && isfinite(fz)) || (fx == 0.0f && fy == 0.0f && fz == 0.0f))
        return 0;
    long long q[3];
    bool certain = pose.fast != 0;
    if (certain) {
#pragma unroll
        for (int r = 0; r < 3; ++r) {
            const float *a = pose.fa + 3 * r;
            const float c = fmaf(a[2], fz, fmaf(a[1], fy, fmaf(a[0], fx, pose.fb[r])));
            const float S = fabsf(a[0] * fx) + fabsf(a[1] * fy) + fabsf(a[2] * fz) + fabsf(pose.fb[r]);
            long long qq = 0;
            certain = certain && floor_certain(c, fmaf(S, FILTER_REL, pose.fe0[r] + FILTER_ABS), qq);
            q[r] = qq + pose.fbi[r];
        }
    }
    const double px = fx, py = fy, pz = fz;
    double d[3];
    bool have_d = false;
    if (!certain) {
        direction64(pose, px, py, pz, d);
        have_d = true;
        const double org[3] = {g.ox, g.oy, g.oz};
#pragma unroll
        for (int r = 0; r < 3; ++r) {
            const double w = __dadd_rn(d[r], pose.t[r]);
            // floor((w - origin) / res) as an integer: the conversion
            // rounds toward -inf and saturates, so the bounds test below is
            // the same as on the binary64 value
            q[r] = __double2ll_rd(__ddiv_rn(__dsub_rn(w, org[r]), g.res));
        }
    }
    if (!(q[0] >= p.R && q[0] <= g.nx - 1 - p.R && q[1] >= p.R && q[1] <= g.ny - 1 - p.R &&
          q[2] >= p.R && q[2] <= g.nz - 1 - p.R))
        return 1;
    int bin = -1;
    if (p.scheme == DBT_BINS_OCTA && pose.fast) {
        float df[3], ef[3];
#pragma unroll
        for (int r = 0; r < 3; ++r) {
            const float *a = pose.fr + 3 * r;
            df[r] = fmaf(a[2], fz, fmaf(a[1], fy, a[0] * fx));
            ef[r] = fmaf(fabsf(a[0] * fx) + fabsf(a[1] * fy) + fabsf(a[2] * fz), FILTER_REL, FILTER_ABS);
        }
        bin = bin_octa_f32(df, ef, p.na);
    }
    if (bin < 0) {
        if (!have_d) direction64(pose, px, py, pz, d);
        bin = bin_of(p, t, d[0], d[1], d[2]);
    }
    rec = make_int4((int)q[0], (int)q[1], (int)q[2], bin);
    return 2;
}

// EX: the update's pre-steps (ScanEx): returns off the downsampling stride
// are not handed in at all, the others use the pose of their time slice.
template <bool EX>
__global__ void __launch_bounds__(256) k_voxelize(DevGrid g, DevParams p, DevTables t, Pose pose,
                                                  const float *__restrict__ xyz, int n, WsDev ws,
                                                  uint32_t hcap, ScanEx ex) {
    __shared__ CtaTally s_tally;
    tally_init(s_tally, 0);
    pdl_wait();
    pdl_launch_dependents();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    bool f[TALLY_FLAGS] = {false, false, false};      // valid, inside, first of its voxel
    int4 rec = make_int4(-1, 0, 0, 0);
    if (i < n) {
        int c = 0;
        if constexpr (EX) {
            if (i % ex.ds == 0) {
                if (ex.n_poses > 0) {
                    const long long m = ((long long)i % ex.period) * ex.n_poses / ex.period;
                    c = contact_of(g, p, t, ws.poses[m], xyz[3 * i + 0], xyz[3 * i + 1], xyz[3 * i + 2], rec);
                } else {
                    c = contact_of(g, p, t, pose, xyz[3 * i + 0], xyz[3 * i + 1], xyz[3 * i + 2], rec);
                }
            }
        } else {
            c = contact_of(g, p, t, pose, xyz[3 * i + 0], xyz[3 * i + 1], xyz[3 * i + 2], rec);
        }
        f[0] = c > 0;
        f[1] = c == 2;
        // the pairs of a contact voxel are counted once, by the insert that
        // created its slot: the kept return's bricks are those of its voxel
        if (f[1]) f[2] = !p.dedup || hash_insert(ws, hcap, voxel_key(g, rec.x, rec.y, rec.z), (uint32_t)i);
        ws.prec[i] = rec;
    }
    count_pairs<true>(ws, g, 0u, f[2], f[2] ? brick_span(rec.x, rec.y, rec.z, p.R, g.bzs) : BrickSpan{});
    tally_warp(s_tally, f);
    tally_flush(s_tally, ws);
}

// Contact voxel and bin of every return (dbt_scan_contacts).
__global__ void __launch_bounds__(256) k_contacts(DevGrid g, DevParams p, DevTables t, Pose pose,
                                                  const float *__restrict__ xyz, long long n,
                                                  int4 *__restrict__ out) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int4 rec = make_int4(-1, 0, 0, 0);
    contact_of(g, p, t, pose, xyz[3 * i + 0], xyz[3 * i + 1], xyz[3 * i + 2], rec);
    out[i] = rec;
}

__device__ __forceinline__ int item_of(const BatchDev &bd, long long i);
__device__ __forceinline__ unsigned long long batch_key(const DevGrid &g, int item, int x, int y,
                                                        int z);

// ------------------------------------------------------------------ K3
// Every brick of the grid(s) is visited: the touched ones (a non-zero pair
// count) get one contiguous segment of the pair array (warp-aggregated bump
// of the pool counter), are counted in n_touched, have their counter reset to
// serve as fill cursor, and are queued for the integrate kernel: heavy
// bricks (more than ws.heavy pairs) for whole CTAs, light ones in their size
// class (light_class), each class claimed by the warps before the next
// smaller one.
// The queue counters are shared by the whole grid, so their bumps are
// aggregated per CTA of 1024 bricks: warp totals are scanned in shared
// memory and one thread takes each counter's range with a single atomic.
constexpr int ALLOC_THREADS = 1024;
constexpr int ALLOC_CTRS = 3 + LIGHT_CLASSES;          // pairs, heavy, very heavy, light classes
// The per-CTA counter scan gives lane j of warp k warp j's entry of counter
// k: one entry per lane, so exactly 32 warps, and a warp per counter.
static_assert(ALLOC_THREADS == 32 * 32 && ALLOC_CTRS <= ALLOC_THREADS / 32,
              "k_alloc's counter scan: 32 warps of 32 lanes, one warp per counter");

// The first-return rule resolved for every return of the scan(s): a kept
// contact that is not its voxel's lowest index is flagged PREC_DUP (grid
// stride over the returns, beside the brick visit below).
template <bool BATCH>
__global__ void __launch_bounds__(ALLOC_THREADS) k_alloc(DevGrid g0, BatchDev bd, DevParams p,
                                                         long long n, WsDev ws, uint32_t hcap) {
    __shared__ uint32_t s_w[ALLOC_THREADS / 32][ALLOC_CTRS];
    __shared__ uint32_t s_tot[ALLOC_CTRS];             // the CTA's total of each counter
    pdl_wait();
    pdl_launch_dependents();
    if (p.dedup) {
        const long long stride = (long long)gridDim.x * ALLOC_THREADS;
        for (long long i = (long long)blockIdx.x * ALLOC_THREADS + threadIdx.x; i < n; i += stride) {
            int4 r = ws.prec[i];
            if (r.x < 0) continue;
            unsigned long long key;
            if constexpr (BATCH) key = batch_key(bd.grids[(r.w >> 16) & 0xFF], item_of(bd, i), r.x, r.y, r.z);
            else key = voxel_key(g0, r.x, r.y, r.z);
            if (!hash_is_first(ws, hcap, key, (uint32_t)i)) {
                r.w |= PREC_DUP;
                ws.prec[i] = r;
            }
        }
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t nb = ws.nbricks;
    for (uint32_t base = blockIdx.x * ALLOC_THREADS; base < nb; base += gridDim.x * ALLOC_THREADS) {
        const uint32_t b = base + threadIdx.x;
        const uint32_t len = b < nb ? ws.bcnt[b] : 0u;
        if (!__syncthreads_or(len != 0u)) continue;        // CTA-uniform
        uint32_t incl = len;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t v = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += v;
        }
        const bool touched = len != 0u;
        const bool heavy = touched && len > ws.heavy;
        const bool vheavy = heavy && len / VHEAVY_FACTOR > ws.heavy;
        // counter index: 1 heavy, 2 very heavy, 3 + c light class c, -1 untouched
        const int cls = !touched ? -1 : vheavy ? 2 : heavy ? 1 : 3 + light_class(len, ws.heavy);
        unsigned bal[ALLOC_CTRS];
#pragma unroll
        for (int k = 1; k < ALLOC_CTRS; ++k) bal[k] = __ballot_sync(0xffffffffu, cls == k);
        if (lane == 31) s_w[warp][0] = incl;
        if (lane == 0) {
#pragma unroll
            for (int k = 1; k < ALLOC_CTRS; ++k) s_w[warp][k] = __popc(bal[k]);
        }
        __syncthreads();
        if (warp < ALLOC_CTRS) {                           // warp k: counter k; lane j: warp j's entry
            const int k = warp;
            const uint32_t v = s_w[lane][k];
            uint32_t x = v;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
                if (lane >= o) x += y;
            }
            uint32_t g = 0u;
            if (lane == 31) {
                s_tot[k] = x;
                if (x) {
                    unsigned int *ctr = k == 0   ? &ws.hdr->pool
                                        : k == 1 ? &ws.hdr->n_heavy
                                        : k == 2 ? &ws.hdr->n_vheavy
                                                 : &ws.hdr->n_cls[k - 3];
                    g = atomicAdd(ctr, x);
                }
            }
            s_w[lane][k] = __shfl_sync(0xffffffffu, g, 31) + x - v;
        }
        __syncthreads();
        if (threadIdx.x == 0) {                            // touched bricks: every class
            uint32_t t = 0u;
#pragma unroll
            for (int k = 1; k < ALLOC_CTRS; ++k) t += s_tot[k];
            if (t) atomicAdd(&ws.hdr->n_touched, t);
        }
        const unsigned below = (1u << lane) - 1u;
        if (touched) {
            ws.boff[b] = s_w[warp][0] + incl - len;
            ws.bcnt[b] = 0;
            const uint32_t q = s_w[warp][cls] + __popc(bal[cls] & below);
            if (q >= ws.max_touched) atomicOr(&ws.hdr->err, ERR_TOUCHED_OVERFLOW);   // cannot happen by sizing
            else if (vheavy) ws.order[ws.max_touched - 1 - q] = b;
            else if (heavy) ws.order[q] = b;
            else *light_queue_slot(ws, cls - 3, q) = b;
        }
        __syncthreads();                                   // s_w is reused next round
    }
}

// ------------------------------------------------------------------ K4
// Pair payload: contact relative to the brick corner plus R (x: 6 bits,
// y, z: 5 bits each) and the bin (16 bits).
__device__ __forceinline__ uint32_t pair_payload(int4 r, int bx, int by, int bz, int R, int bzs) {
    const uint32_t rx = (uint32_t)(r.x - bx * BX + R);
    const uint32_t ry = (uint32_t)(r.y - by * BY + R);
    const uint32_t rz = (uint32_t)(r.z - (bz << bzs) + R);
    return rx | (ry << 6) | (rz << 11) | ((uint32_t)(r.w & 0xFFFF) << 16);
}

// Pair payloads into the segments, slots from the per-brick cursors.  One
// thread per (return, block of FILL_UNROLL consecutive bricks of its span):
// grid row y = blockIdx.y takes bricks j = y * FILL_UNROLL ... of the spans
// (x fastest), returns along x; with a single grid row a thread takes its
// whole span, FILL_UNROLL bricks at a time.  A warp walks its 32 returns'
// bricks j in lock-step, and the lanes that name one brick take their slots
// with one atomic of their leader (the j-th bricks of consecutive returns
// mostly coincide).  The FILL_UNROLL bricks of a block are issued together --
// their cursor atomics and segment-offset loads are all in flight before
// the first result is used -- so a thread waits once per block.  b0: first
// brick index of the return's grid (batches).
constexpr int FILL_UNROLL = 4;
static_assert(MAX_K - 1 <= BX && MAX_K - 1 <= 3 * BY, "fill_span's decomposition: sx <= 2, sy <= 4");
__device__ __forceinline__ void fill_span(bool has, int4 r, const DevGrid &g, uint32_t b0, int R,
                                          const WsDev &ws) {
    const BrickSpan sp = has ? brick_span(r.x, r.y, r.z, R, g.bzs) : BrickSpan{};
    const int sx = sp.x1 - sp.x0 + 1, sy = sp.y1 - sp.y0 + 1, sz = sp.z1 - sp.z0 + 1;
    const int np = has ? sx * sy * sz : 0;
    const int jbeg = (int)blockIdx.y * FILL_UNROLL;
    const int jend = gridDim.y == 1 ? np : jbeg + FILL_UNROLL;
    const int nsteps = __reduce_max_sync(0xffffffffu, min(np, jend));
    const int lane = threadIdx.x & 31;
    const unsigned below = (1u << lane) - 1u;
    for (int j0 = jbeg; j0 < nsteps; j0 += FILL_UNROLL) {
        uint32_t b[FILL_UNROLL], pl[FILL_UNROLL], old[FILL_UNROLL], off[FILL_UNROLL];
        unsigned peers[FILL_UNROLL];
#pragma unroll
        for (int u = 0; u < FILL_UNROLL; ++u) {
            const int j = j0 + u;
            b[u] = 0xFFFFFFFFu;                      // no brick (never a brick index: < 2^32 - 1 bricks)
            pl[u] = 0u;
            if (j < np) {
                // j -> (ix, iy, iz), x fastest; sx <= 2 and sy <= 4 for K <= 21
                const int ix = sx == 1 ? 0 : (j & 1);
                int iy = sx == 1 ? j : (j >> 1), iz = 0;
                while (iy >= sy) {
                    iy -= sy;
                    ++iz;
                }
                const int bx = sp.x0 + ix, by = sp.y0 + iy, bz = sp.z0 + iz;
                b[u] = b0 + ((uint32_t)bz * g.nby + by) * g.nbx + bx;
                pl[u] = pair_payload(r, bx, by, bz, R, g.bzs);
            }
            peers[u] = __match_any_sync(0xffffffffu, b[u]);
            old[u] = 0u;
            off[u] = 0u;
            if (b[u] != 0xFFFFFFFFu) {
                if (lane == __ffs(peers[u]) - 1) old[u] = atomicAdd(&ws.bcnt[b[u]], (uint32_t)__popc(peers[u]));
                off[u] = ws.boff[b[u]];
            }
        }
#pragma unroll
        for (int u = 0; u < FILL_UNROLL; ++u) {
            const uint32_t base = __shfl_sync(0xffffffffu, old[u], __ffs(peers[u]) - 1);
            if (b[u] != 0xFFFFFFFFu) {
                const unsigned long long pos =
                    (unsigned long long)off[u] + base + (uint32_t)__popc(peers[u] & below);
                if (pos < ws.pairs_cap) ws.pairs[pos] = pl[u];
                else atomicOr(&ws.hdr->err, ERR_PAIRS_OVERFLOW);
            }
        }
    }
}

// Clears the first-return hash table for the next scan (grid stride over
// every thread of the 2-D grid).
__device__ __forceinline__ void clear_hash(const WsDev &ws, uint32_t hcap) {
    const unsigned long long stride = (unsigned long long)gridDim.x * gridDim.y * blockDim.x;
    for (unsigned long long k = ((unsigned long long)blockIdx.y * gridDim.x + blockIdx.x) * blockDim.x +
                                threadIdx.x;
         k < hcap; k += stride) {
        ws.hkey[k] = 0ull;
        ws.hidx[k] = 0u;
    }
}

__global__ void __launch_bounds__(256) k_fill(DevGrid g, DevParams p, int n, WsDev ws, uint32_t hcap) {
    pdl_wait();
    pdl_launch_dependents();
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    int4 r = make_int4(-1, 0, 0, 0);
    if (i < n) r = ws.prec[i];
    fill_span(r.x >= 0 && !(r.w & PREC_DUP), r, g, 0u, p.R, ws);
    if (p.dedup) clear_hash(ws, hcap);
}

// ------------------------------------------------------------------ batches
// The same stages for every scan of a batch at once.  Returns of all scans
// share one index space (scan k owns [istart[k], istart[k+1])); the
// first-return hash key carries the scan, so the rule stays per scan; bricks
// of all grids share one index space (grid m owns [bbase[m], bbase[m+1])).

__device__ __forceinline__ int item_of(const BatchDev &bd, long long i) {
    int lo = 0, hi = bd.n_items - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (bd.istart[mid] <= i) lo = mid; else hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ unsigned long long batch_key(const DevGrid &g, int item, int x, int y,
                                                        int z) {
    return ((unsigned long long)item << 40) + voxel_key(g, x, y, z);
}

// Adds per-scan counts of a warp (valid, inside, kept): lanes with the same
// item are summed by their leader, into the CTA's window (or directly past
// it).
__device__ __forceinline__ void add_item_counts(const BatchDev &bd, CtaTally &s, int item,
                                                const bool f[TALLY_FLAGS]) {
    const unsigned peers = __match_any_sync(0xffffffffu, item);
    unsigned bal[TALLY_FLAGS];
#pragma unroll
    for (int k = 0; k < TALLY_FLAGS; ++k) bal[k] = __ballot_sync(0xffffffffu, f[k]) & peers;
    const int lane = threadIdx.x & 31;
    if (item >= 0 && lane == __ffs(peers) - 1) {
        const int w = item - s.first_item;
        unsigned long long *g[TALLY_FLAGS] = {&bd.icnt[item].valid, &bd.icnt[item].inside,
                                             &bd.icnt[item].kept};
#pragma unroll
        for (int k = 0; k < TALLY_FLAGS; ++k) {
            if (!bal[k]) continue;
            if (w >= 0 && w < TALLY_ITEMS) atomicAdd(&s.item[w][k], (uint32_t)__popc(bal[k]));
            else atomicAdd(g[k], (unsigned long long)__popc(bal[k]));
        }
    }
}

// The CTA's per-scan window to the global per-scan counters (after
// tally_flush's barrier).
__device__ __forceinline__ void flush_item_counts(const BatchDev &bd, CtaTally &s) {
    const int w = threadIdx.x;
    if (w < TALLY_ITEMS && s.first_item >= 0 && s.first_item + w < bd.n_items) {
        ItemCounters &c = bd.icnt[s.first_item + w];
        if (s.item[w][0]) atomicAdd(&c.valid, (unsigned long long)s.item[w][0]);
        if (s.item[w][1]) atomicAdd(&c.inside, (unsigned long long)s.item[w][1]);
        if (s.item[w][2]) atomicAdd(&c.kept, (unsigned long long)s.item[w][2]);
    }
}

// First scan of the CTA's returns (-1 when it has none).
__device__ __forceinline__ int cta_first_item(const BatchDev &bd, long long n) {
    const long long i0 = (long long)blockIdx.x * blockDim.x;
    return i0 < n ? item_of(bd, i0) : -1;
}

__global__ void __launch_bounds__(256) k_voxelize_b(BatchDev bd, DevParams p, DevTables t,
                                                    long long n, WsDev ws, uint32_t hcap) {
    __shared__ CtaTally s_tally;
    pdl_wait();
    pdl_launch_dependents();
    tally_init(s_tally, threadIdx.x == 0 ? cta_first_item(bd, n) : 0);
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    bool f[TALLY_FLAGS] = {false, false, false};      // valid, inside, first of its voxel
    int item = -1;
    int4 rec = make_int4(-1, 0, 0, 0);
    DevGrid g = {};
    uint32_t b0 = 0;
    if (i < n) {
        item = item_of(bd, i);
        const ItemDev &it = bd.items[item];
        g = bd.grids[it.grid];
        b0 = bd.bbase[it.grid];
        const long long j = i - bd.istart[item];
        const int c = contact_of(g, p, t, it.pose, it.xyz[3 * j + 0], it.xyz[3 * j + 1],
                                 it.xyz[3 * j + 2], rec);
        f[0] = c > 0;
        f[1] = c == 2;
        if (f[1]) {
            f[2] = !p.dedup || hash_insert(ws, hcap, batch_key(g, item, rec.x, rec.y, rec.z), (uint32_t)i);
            ws.prec[i] = make_int4(rec.x, rec.y, rec.z, rec.w | (it.grid << 16));
        } else {
            ws.prec[i] = rec;
        }
    }
    count_pairs<true>(ws, g, b0, f[2], f[2] ? brick_span(rec.x, rec.y, rec.z, p.R, g.bzs) : BrickSpan{});
    tally_warp(s_tally, f);
    add_item_counts(bd, s_tally, item, f);
    tally_flush(s_tally, ws);
    flush_item_counts(bd, s_tally);
}

// The same for the returns of all scans of a batch (each return in its
// grid's brick range).
__global__ void __launch_bounds__(256) k_fill_b(BatchDev bd, DevParams p, long long n, WsDev ws,
                                                uint32_t hcap) {
    pdl_wait();
    pdl_launch_dependents();
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    int4 r = make_int4(-1, 0, 0, 0);
    if (i < n) r = ws.prec[i];
    const bool has = r.x >= 0 && !(r.w & PREC_DUP);
    DevGrid g = {};
    uint32_t b0 = 0;
    if (has) {
        const int gi = (r.w >> 16) & 0xFF;
        g = bd.grids[gi];
        b0 = bd.bbase[gi];
    }
    fill_span(has, r, g, b0, p.R, ws);
    if (p.dedup) clear_hash(ws, hcap);
}

// ------------------------------------------------------------------ footprint
// Measurement pass (not part of integration): marks, in two caller-owned
// bitmaps over the padded grid, every voxel of a kept return's K^3
// neighbourhood and of its shadow set, and counts first-time marks.  The
// counts U and U_s give the algorithmic bytes of a scan's integration.
__global__ void __launch_bounds__(256) k_footprint(DevGrid g, DevParams p, DevTables t, int n,
                                                   uint32_t hcap,
                                                   WsDev ws, uint32_t *bits_u, uint32_t *bits_s,
                                                   unsigned long long *counts) {
    const int i = blockIdx.x;
    if (i >= n) return;
    const int4 r = ws.prec[i];
    if (r.x < 0) return;
    if (p.dedup && !hash_is_first(ws, hcap, voxel_key(g, r.x, r.y, r.z), (uint32_t)i)) return;
    const int R = p.R, K = p.K;
    unsigned long long nu = 0, ns = 0;
    for (int e = threadIdx.x; e < K * K * K; e += blockDim.x) {
        const int ox = e % K - R, oy = (e / K) % K - R, oz = e / (K * K) - R;
        const unsigned long long v = voxel_key(g, r.x + ox, r.y + oy, r.z + oz) - 1ull;
        const uint32_t bit = 1u << (v & 31);
        if (!(atomicOr(&bits_u[v >> 5], bit) & bit)) ++nu;
    }
    const uint32_t bin = (uint32_t)(r.w & 0xFFFF);
    for (uint32_t e = t.sh_start[bin] + threadIdx.x; e < t.sh_start[bin + 1]; e += blockDim.x) {
        const uint32_t o = t.sh_off[e];
        const unsigned long long v =
            voxel_key(g, r.x + off_axis(o, 0), r.y + off_axis(o, 1), r.z + off_axis(o, 2)) - 1ull;
        const uint32_t bit = 1u << (v & 31);
        if (!(atomicOr(&bits_s[v >> 5], bit) & bit)) ++ns;
    }
    if (nu) atomicAdd(&counts[0], nu);
    if (ns) atomicAdd(&counts[1], ns);
}

// Returns the workspace to its between-scans state after k_voxelize ran
// without the rest of the pipeline (brick counters, hash table, header).
__global__ void k_ws_rearm(WsDev ws, uint32_t hcap) {
    const uint32_t stride = gridDim.x * blockDim.x;
    const uint32_t g0 = blockIdx.x * blockDim.x + threadIdx.x;
    for (uint32_t j = g0; j < ws.nbricks; j += stride) ws.bcnt[j] = 0u;   // every brick counter
    for (uint32_t j = g0; j < hcap; j += stride) {
        ws.hkey[j] = 0ull;
        ws.hidx[j] = 0u;
    }
}

__global__ void k_ws_rearm_header(WsDev ws) {
    WsHeader *h = ws.hdr;
    h->err = 0u;
    h->n_touched = 0u;
    h->pool = 0u;
    h->next_work = 0u;
    h->done_ctas = 0u;
    h->n_heavy = 0u;
    h->n_vheavy = 0u;
    for (int c = 0; c < LIGHT_CLASSES; ++c) h->n_cls[c] = 0u;
    h->next_heavy = 0u;
    h->next_vheavy = 0u;
    h->acc_valid = 0ull;
    h->acc_inside = 0ull;
    h->acc_kept = 0ull;
}

void launch_footprint(const DevGrid &g, const DevParams &p, const DevTables &t, int n,
                      const WsDev &ws, uint32_t hcap, uint32_t *bits_u, uint32_t *bits_s,
                      unsigned long long *counts, cudaStream_t s) {
    if (n > 0) k_footprint<<<n, 256, 0, s>>>(g, p, t, n, hcap, ws, bits_u, bits_s, counts);
    k_ws_rearm<<<2 * device_sm_count(), 256, 0, s>>>(ws, hcap);
    k_ws_rearm_header<<<1, 1, 0, s>>>(ws);
}

// ------------------------------------------------------------------ readouts
__global__ void k_bin_dirs(DevParams p, DevTables t, const double *__restrict__ dirs, int n,
                           int *__restrict__ bins) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double x = dirs[3 * i], y = dirs[3 * i + 1], z = dirs[3 * i + 2];
    bins[i] = (x == 0.0 && y == 0.0 && z == 0.0) ? -1 : bin_of(p, t, x, y, z);
}

__global__ void k_read_voxels(DevGrid g, const int *__restrict__ idx, long long n,
                              uint32_t *__restrict__ mask, uint8_t *__restrict__ sign,
                              uint16_t *__restrict__ hits) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int x = idx[3 * i], y = idx[3 * i + 1], z = idx[3 * i + 2];
    uint32_t m = 0xFFFFFFFFu;
    uint8_t s = 1;
    uint16_t h = 0;
    if (x >= 0 && x < g.nx && y >= 0 && y < g.ny && z >= 0 && z < g.nz) {
        const size_t v = ((size_t)z * g.ny + y) * g.pitch + x;
        m = g.mask[v];
        s = g.sign[v];
        h = g.hits[v];
    }
    if (mask) mask[i] = m;
    if (sign) sign[i] = s;
    if (hits) hits[i] = h;
}

__global__ void k_read_distance(DevGrid g, double res, const int *__restrict__ idx, long long n,
                                float *__restrict__ sdf) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int x = idx[3 * i], y = idx[3 * i + 1], z = idx[3 * i + 2];
    uint32_t m = 0xFFFFFFFFu;
    uint8_t s = 1;
    if (x >= 0 && x < g.nx && y >= 0 && y < g.ny && z >= 0 && z < g.nz) {
        const size_t v = ((size_t)z * g.ny + y) * g.pitch + x;
        m = g.mask[v];
        s = g.sign[v];
    }
    const double d = (double)__popc(m) * res;
    sdf[i] = (float)(s ? d : -d);
}

// ------------------------------------------------------------------ launchers
static inline int blocks_for(long long n, int tpb) { return (int)((n + tpb - 1) / tpb); }

void launch_voxelize(const DevGrid &g, const DevParams &p, const DevTables &t, const Pose &pose,
                     const float *xyz, int n, const WsDev &ws, uint32_t hcap, cudaStream_t s,
                     const ScanEx *ex) {
    if (ex)
        launch_pdl(k_voxelize<true>, max(1, blocks_for(n, 256)), 256, 0, s, g, p, t, pose, xyz, n, ws,
                   hcap, *ex);
    else
        launch_pdl(k_voxelize<false>, max(1, blocks_for(n, 256)), 256, 0, s, g, p, t, pose, xyz, n, ws,
                   hcap, ScanEx{1, 0, 1});
}

void launch_contacts(const DevGrid &g, const DevParams &p, const DevTables &t, const Pose &pose,
                     const float *xyz, long long n, int4 *out, cudaStream_t s) {
    if (n > 0) k_contacts<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(g, p, t, pose, xyz, n, out);
}

// One thread per brick where the GPU holds them all at once (a single wave
// hides the latency of the counter loads and queue atomics), grid-stride
// beyond that; the first-return resolve strides over the returns.
static int alloc_ctas(long long nbricks, long long n) {
    const long long need = (std::max(nbricks, n) + ALLOC_THREADS - 1) / ALLOC_THREADS;
    return (int)std::max(1LL, std::min(need, 4LL * device_sm_count()));
}

void launch_alloc(const DevGrid &g, const DevParams &p, long long n, const WsDev &ws, uint32_t hcap,
                  cudaStream_t s) {
    launch_pdl(k_alloc<false>, alloc_ctas(ws.nbricks, n), ALLOC_THREADS, 0, s, g, BatchDev{}, p, n, ws,
               hcap);
}

void launch_alloc_batch(const BatchDev &bd, const DevParams &p, long long n, const WsDev &ws,
                        uint32_t hcap, cudaStream_t s) {
    launch_pdl(k_alloc<true>, alloc_ctas(ws.nbricks, n), ALLOC_THREADS, 0, s, DevGrid{}, bd, p, n, ws,
               hcap);
}

// Grid rows of the fill: one when a thread per return already fills the
// GPU several times over (large batches: more rows would only add waves),
// else blocks of FILL_UNROLL bricks of the longest span.
static unsigned fill_rows(long long n, const DevParams &p, int bz) {
    if (n >= 2048ll * device_sm_count()) return 1u;
    return (unsigned)((max_pairs_per_return(p.K, bz) + FILL_UNROLL - 1) / FILL_UNROLL);
}

void launch_fill(const DevGrid &g, const DevParams &p, int n, const WsDev &ws, uint32_t hcap,
                 cudaStream_t s) {
    launch_pdl(k_fill, dim3((unsigned)std::max(1, (n + 255) / 256), fill_rows(n, p, 1 << g.bzs)), 256, 0, s,
               g, p, n, ws, hcap);
}

static inline unsigned batch_blocks(long long n) { return (unsigned)max(1ll, (n + 255) / 256); }

void launch_voxelize_batch(const BatchDev &bd, const DevParams &p, const DevTables &t,
                           long long n, const WsDev &ws, uint32_t hcap, cudaStream_t s) {
    launch_pdl(k_voxelize_b, batch_blocks(n), 256, 0, s, bd, p, t, n, ws, hcap);
}

void launch_fill_batch(const BatchDev &bd, const DevParams &p, long long n, const WsDev &ws,
                       uint32_t hcap, cudaStream_t s) {
    launch_pdl(k_fill_b, dim3(batch_blocks(n), fill_rows(n, p, 1 << bd.bzs)), 256, 0, s, bd, p, n, ws, hcap);
}

void launch_bin_dirs(const DevParams &p, const DevTables &t, const double *dirs, int n, int *bins,
                     cudaStream_t s) {
    if (n > 0) k_bin_dirs<<<blocks_for(n, 256), 256, 0, s>>>(p, t, dirs, n, bins);
}

void launch_read_voxels(const DevGrid &g, const int *idx, long long n, uint32_t *mask,
                        uint8_t *sign, uint16_t *hits, cudaStream_t s) {
    if (n > 0) k_read_voxels<<<blocks_for(n, 256), 256, 0, s>>>(g, idx, n, mask, sign, hits);
}

void launch_read_distance(const DevGrid &g, double res, const int *idx, long long n, float *sdf,
                          cudaStream_t s) {
    if (n > 0) k_read_distance<<<blocks_for(n, 256), 256, 0, s>>>(g, res, idx, n, sdf);
}

}  // namespace dbt
