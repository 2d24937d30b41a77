// Reconstruction quality (Sec. IV-B, "Mapping results"): exact nearest-
// neighbour distances between a predicted point set (sampled from the
// reconstructed mesh's iso-surface) and reference surface points, and the
// metrics built on them: accuracy (mean predicted -> reference distance),
// completeness (mean reference -> predicted), Chamfer-L1 (their mean),
// precision / recall (fractions within the tolerance, d < t) and F-score.
//
// Index: the reference points are counting-sorted into a uniform grid of
// about 4 cells per point over the bounding box of both sets, with a coarse
// occupancy count per block of 8 x 8 x 8 cells.  A query visits rings of
// cells at Chebyshev distance k = 0, 1, 2 around its own cell and stops
// after ring k once its best distance is at most (k - 1/100) h: every point
// outside the rings already seen is at least k h away (the 1 % slack covers
// the rounding of the cell assignment).  Queries still open then walk rings
// of blocks (edge H = 8 h), skipping empty blocks, with the same rule on H,
// so far-away queries cost (D / H)^3 block tests instead of (D / h)^3 cell
// visits.  The result is the exact minimum; distances are evaluated in
// binary32.
#include "dbt_internal.cuh"

namespace dbt {

namespace {

struct NnHeader {
    uint32_t lo_key[3], hi_key[3];     // order-preserving float keys of the bounds
    float lo[3];
    float h, inv_h;
    int dims[3];
    int cdims[3];                      // blocks of 8 x 8 x 8 cells
    unsigned long long ncell;
    unsigned long long total;
};

constexpr int kBlock = 8;

constexpr int kNnTarget = 4;                     // cells per reference point
constexpr unsigned long long kNnMaxCells = 1ull << 25;

__host__ __device__ inline unsigned long long nn_cells_for(long long n_ref) {
    const unsigned long long c = (unsigned long long)(n_ref > 0 ? n_ref : 1) * kNnTarget;
    return c < kNnMaxCells ? c : kNnMaxCells;
}

__device__ __forceinline__ uint32_t fkey(float f) {
    const uint32_t b = __float_as_uint(f);
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}
__device__ __forceinline__ float fval(uint32_t k) {
    return __uint_as_float((k & 0x80000000u) ? (k & 0x7FFFFFFFu) : ~k);
}

struct NnLayout {
    NnHeader *hdr;
    uint32_t *bcnt;                // points per block (<= budget / 8 + 1 blocks)
    uint32_t *cnt;                 // ncell + 1 (counts, then fill cursors)
    unsigned long long *off;       // ncell + 1 exclusive offsets
    unsigned long long *tile;      // scan partials
    float4 *pts;                   // reference points by cell
    size_t bytes;
};

size_t up256(size_t x) { return (x + 255) & ~size_t(255); }

NnLayout nn_layout(long long n_ref, void *scratch) {
    const unsigned long long C = nn_cells_for(n_ref) + 1;
    const unsigned long long nt = (C + 1023) / 1024;
    char *p = static_cast<char *>(scratch);
    size_t o = 0;
    NnLayout L{};
    L.hdr = reinterpret_cast<NnHeader *>(p + o);
    o += up256(sizeof(NnHeader));
    L.bcnt = reinterpret_cast<uint32_t *>(p + o);
    o += up256((C / kBlock + 2) * 4);
    L.cnt = reinterpret_cast<uint32_t *>(p + o);
    o += up256(C * 4);
    L.off = reinterpret_cast<unsigned long long *>(p + o);
    o += up256(C * 8);
    L.tile = reinterpret_cast<unsigned long long *>(p + o);
    o += up256(nt * 8);
    L.pts = reinterpret_cast<float4 *>(p + o);
    o += up256((size_t)(n_ref > 0 ? n_ref : 1) * 16);
    L.bytes = o;
    return L;
}

__global__ void k_nn_init(NnHeader *h) {
    for (int a = 0; a < 3; ++a) {
        h->lo_key[a] = 0xFFFFFFFFu;
        h->hi_key[a] = 0u;
    }
}

__global__ void __launch_bounds__(256) k_nn_bounds(const float *__restrict__ a, long long na,
                                                   const float *__restrict__ b, long long nb,
                                                   NnHeader *h) {
    uint32_t lo[3] = {0xFFFFFFFFu, 0xFFFFFFFFu, 0xFFFFFFFFu}, hi[3] = {0u, 0u, 0u};
    const long long n = na + nb;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const float *p = i < na ? a + 3 * i : b + 3 * (i - na);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const uint32_t k = fkey(p[c]);
            lo[c] = min(lo[c], k);
            hi[c] = max(hi[c], k);
        }
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        lo[c] = __reduce_min_sync(0xffffffffu, lo[c]);
        hi[c] = __reduce_max_sync(0xffffffffu, hi[c]);
    }
    if ((threadIdx.x & 31) == 0)
        for (int c = 0; c < 3; ++c) {
            atomicMin(&h->lo_key[c], lo[c]);
            atomicMax(&h->hi_key[c], hi[c]);
        }
}

// Cell edge h from the box volume and the cell budget; dims = ceil(ext / h).
__global__ void k_nn_setup(NnHeader *h, unsigned long long budget) {
    float lo[3], ext[3], emax = 0.f;
    for (int a = 0; a < 3; ++a) {
        lo[a] = fval(h->lo_key[a]);
        const float hi = fval(h->hi_key[a]);
        ext[a] = h->lo_key[a] <= h->hi_key[a] ? hi - lo[a] : 0.f;
        emax = fmaxf(emax, ext[a]);
        h->lo[a] = h->lo_key[a] <= h->hi_key[a] ? lo[a] : 0.f;
    }
    const float floor_e = emax > 0.f ? emax * 1e-3f : 1.f;
    const double vol = (double)fmaxf(ext[0], floor_e) * fmaxf(ext[1], floor_e) * fmaxf(ext[2], floor_e);
    float cell = (float)cbrt(vol / (double)budget);
    unsigned long long n = 0;
    for (int it = 0; it < 64; ++it) {               // grow h until the grid fits the budget
        n = 1;
        for (int a = 0; a < 3; ++a) n *= (unsigned long long)(floorf(ext[a] / cell) + 1.f);
        if (n <= budget) break;
        cell *= 1.05f;
    }
    h->h = cell;
    h->inv_h = 1.f / cell;
    for (int a = 0; a < 3; ++a) {
        h->dims[a] = (int)(floorf(ext[a] / cell) + 1.f);
        h->cdims[a] = (h->dims[a] + kBlock - 1) / kBlock;
    }
    h->ncell = (unsigned long long)h->dims[0] * h->dims[1] * h->dims[2];
}

__device__ __forceinline__ int nn_axis_cell(float v, float lo, float inv_h, int dim) {
    const int c = (int)floorf((v - lo) * inv_h);
    return c < 0 ? 0 : (c >= dim ? dim - 1 : c);
}

__device__ __forceinline__ long long nn_cell(const NnHeader &h, const float *p) {
    const int cx = nn_axis_cell(p[0], h.lo[0], h.inv_h, h.dims[0]);
    const int cy = nn_axis_cell(p[1], h.lo[1], h.inv_h, h.dims[1]);
    const int cz = nn_axis_cell(p[2], h.lo[2], h.inv_h, h.dims[2]);
    return ((long long)cz * h.dims[1] + cy) * h.dims[0] + cx;
}

__global__ void __launch_bounds__(256) k_nn_count(const float *__restrict__ ref, long long n,
                                                  const NnHeader *h, uint32_t *cnt,
                                                  uint32_t *bcnt) {
    const NnHeader hh = *h;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const float *p = ref + 3 * i;
        const int cx = nn_axis_cell(p[0], hh.lo[0], hh.inv_h, hh.dims[0]);
        const int cy = nn_axis_cell(p[1], hh.lo[1], hh.inv_h, hh.dims[1]);
        const int cz = nn_axis_cell(p[2], hh.lo[2], hh.inv_h, hh.dims[2]);
        atomicAdd(&cnt[((long long)cz * hh.dims[1] + cy) * hh.dims[0] + cx], 1u);
        atomicAdd(&bcnt[((long long)(cz / kBlock) * hh.cdims[1] + cy / kBlock) * hh.cdims[0] +
                        cx / kBlock], 1u);
    }
}

__global__ void __launch_bounds__(256) k_nn_scatter(const float *__restrict__ ref, long long n,
                                                    const NnHeader *h,
                                                    const unsigned long long *__restrict__ off,
                                                    uint32_t *cur, float4 *pts) {
    const NnHeader hh = *h;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const float *p = ref + 3 * i;
        const long long c = nn_cell(hh, p);
        const unsigned long long slot = off[c] + atomicAdd(&cur[c], 1u);
        pts[slot] = make_float4(p[0], p[1], p[2], 0.f);
    }
}

// Minimum squared distance from q to the points of cells [x0, x1] of row
// (y, z) -- one call per row segment.
__device__ __forceinline__ float nn_scan_row(const NnHeader &hh, const unsigned long long *off,
                                             const float4 *pts, float qx, float qy, float qz,
                                             int y, int z, int x0, int x1, float best) {
    const long long c0 = ((long long)z * hh.dims[1] + y) * hh.dims[0];
    const unsigned long long e = off[c0 + x1 + 1];
    for (unsigned long long j = off[c0 + x0]; j < e; ++j) {     // the row's cells are contiguous
        const float4 p = pts[j];
        const float dx = __fsub_rn(qx, p.x), dy = __fsub_rn(qy, p.y), dz = __fsub_rn(qz, p.z);
        const float d2 = __fadd_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)), __fmul_rn(dz, dz));
        best = fminf(best, d2);
    }
    return best;
}

__global__ void __launch_bounds__(256) k_nn_query(const float *__restrict__ q, long long n,
                                                  const NnHeader *h,
                                                  const unsigned long long *__restrict__ off,
                                                  const uint32_t *__restrict__ bcnt,
                                                  const float4 *__restrict__ pts,
                                                  float *__restrict__ dist) {
    const NnHeader hh = *h;
    const int kfine = 2;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const float qx = q[3 * i], qy = q[3 * i + 1], qz = q[3 * i + 2];
        const int cx = nn_axis_cell(qx, hh.lo[0], hh.inv_h, hh.dims[0]);
        const int cy = nn_axis_cell(qy, hh.lo[1], hh.inv_h, hh.dims[1]);
        const int cz = nn_axis_cell(qz, hh.lo[2], hh.inv_h, hh.dims[2]);
        float best = __int_as_float(0x7f800000);   // +inf
        bool done = false;
        for (int k = 0; k <= kfine && !done; ++k) {
            const int z0 = max(cz - k, 0), z1 = min(cz + k, hh.dims[2] - 1);
            const int y0 = max(cy - k, 0), y1 = min(cy + k, hh.dims[1] - 1);
            const int x0 = max(cx - k, 0), x1 = min(cx + k, hh.dims[0] - 1);
            for (int z = z0; z <= z1; ++z)
                for (int y = y0; y <= y1; ++y) {
                    if (abs(z - cz) == k || abs(y - cy) == k) {          // a whole row of the ring
                        best = nn_scan_row(hh, off, pts, qx, qy, qz, y, z, x0, x1, best);
                    } else {                                             // its two end cells
                        if (cx - k >= 0) best = nn_scan_row(hh, off, pts, qx, qy, qz, y, z, cx - k, cx - k, best);
                        if (cx + k < hh.dims[0]) best = nn_scan_row(hh, off, pts, qx, qy, qz, y, z, cx + k, cx + k, best);
                    }
                }
            const float reach = ((float)k - 0.01f) * hh.h;
            done = k > 0 && best <= reach * reach;
        }
        if (!done) {
            // rings of non-empty blocks around the query's block, edge H = 8 h
            const int bx = cx / kBlock, by = cy / kBlock, bz = cz / kBlock;
            const int kmax = max(hh.cdims[0], max(hh.cdims[1], hh.cdims[2]));
            const float H = hh.h * (float)kBlock;
            for (int k = 0; k <= kmax; ++k) {
                const int z0 = max(bz - k, 0), z1 = min(bz + k, hh.cdims[2] - 1);
                const int y0 = max(by - k, 0), y1 = min(by + k, hh.cdims[1] - 1);
                const int x0 = max(bx - k, 0), x1 = min(bx + k, hh.cdims[0] - 1);
                for (int z = z0; z <= z1; ++z)
                    for (int y = y0; y <= y1; ++y) {
                        const bool face = abs(z - bz) == k || abs(y - by) == k;
                        for (int x = x0; x <= x1; ++x) {
                            if (!face && abs(x - bx) != k) {
                                if (x < bx + k) x = bx + k - 1;
                                continue;
                            }
                            if (!bcnt[((long long)z * hh.cdims[1] + y) * hh.cdims[0] + x]) continue;
                            const int fz1 = min(z * kBlock + kBlock, hh.dims[2]) - 1;
                            const int fy1 = min(y * kBlock + kBlock, hh.dims[1]) - 1;
                            const int fx0 = x * kBlock, fx1 = min(fx0 + kBlock, hh.dims[0]) - 1;
                            for (int fz = z * kBlock; fz <= fz1; ++fz)
                                for (int fy = y * kBlock; fy <= fy1; ++fy)
                                    best = nn_scan_row(hh, off, pts, qx, qy, qz, fy, fz, fx0, fx1, best);
                        }
                    }
                const float reach = ((float)k - 0.01f) * H;
                if (k > 0 && best <= reach * reach) break;
            }
        }
        dist[i] = sqrtf(best);
    }
}

// ------------------------------------------------------------------ metrics
constexpr int kRedBlocks = 304;
constexpr int kRedThreads = 256;

struct RedPart {
    double s_pred, s_gt;
    unsigned long long in_pred, in_gt;
};

// Fixed grid and fixed per-thread order, then one block sums the block
// partials in order: the result is the same on every run.
__global__ void __launch_bounds__(kRedThreads) k_quality_partials(
    const float *__restrict__ dp, long long np, const float *__restrict__ dg, long long ng,
    float tol, RedPart *part) {
    __shared__ RedPart s[kRedThreads];
    RedPart r = {0.0, 0.0, 0ull, 0ull};
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < np;
         i += (long long)gridDim.x * blockDim.x) {
        r.s_pred += (double)dp[i];
        r.in_pred += dp[i] < tol;
    }
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < ng;
         i += (long long)gridDim.x * blockDim.x) {
        r.s_gt += (double)dg[i];
        r.in_gt += dg[i] < tol;
    }
    s[threadIdx.x] = r;
    __syncthreads();
    for (int w = kRedThreads / 2; w; w >>= 1) {
        if (threadIdx.x < w) {
            s[threadIdx.x].s_pred += s[threadIdx.x + w].s_pred;
            s[threadIdx.x].s_gt += s[threadIdx.x + w].s_gt;
            s[threadIdx.x].in_pred += s[threadIdx.x + w].in_pred;
            s[threadIdx.x].in_gt += s[threadIdx.x + w].in_gt;
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = s[0];
}

__global__ void k_quality_final(const RedPart *part, long long np, long long ng, double *out) {
    RedPart r = {0.0, 0.0, 0ull, 0ull};
    for (int b = 0; b < kRedBlocks; ++b) {
        r.s_pred += part[b].s_pred;
        r.s_gt += part[b].s_gt;
        r.in_pred += part[b].in_pred;
        r.in_gt += part[b].in_gt;
    }
    const double acc = np ? r.s_pred / (double)np : 0.0;
    const double comp = ng ? r.s_gt / (double)ng : 0.0;
    const double prec = np ? (double)r.in_pred / (double)np : 0.0;
    const double rec = ng ? (double)r.in_gt / (double)ng : 0.0;
    out[0] = acc;
    out[1] = comp;
    out[2] = (acc + comp) / 2.0;
    out[3] = prec;
    out[4] = rec;
    out[5] = prec + rec > 0.0 ? 2.0 * prec * rec / (prec + rec) : 0.0;
}

__global__ void __launch_bounds__(256) k_centroids(const float *__restrict__ tri, long long n,
                                                   float *__restrict__ out) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const float *t = tri + 9 * i;
#pragma unroll
        for (int c = 0; c < 3; ++c)
            out[3 * i + c] = __fdiv_rn(__fadd_rn(__fadd_rn(t[c], t[3 + c]), t[6 + c]), 3.0f);
    }
}

__global__ void k_fill_inf(float *d, long long n) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        d[i] = __int_as_float(0x7f800000);
}

int blocks_for(long long n) {
    const long long b = (n + 255) / 256;
    return (int)std::max(1LL, std::min(b, 8LL * device_sm_count()));
}

}  // namespace

size_t nn_scratch_bytes(long long n_ref) { return nn_layout(n_ref, nullptr).bytes; }

void launch_nn_distances(const float *ref, long long n_ref, const float *q, long long n_q,
                         void *scratch, float *dist, cudaStream_t s) {
    if (n_q <= 0) return;
    if (n_ref <= 0) {                                   // no reference point: +inf everywhere
        k_fill_inf<<<blocks_for(n_q), 256, 0, s>>>(dist, n_q);
        return;
    }
    const NnLayout L = nn_layout(n_ref, scratch);
    const unsigned long long budget = nn_cells_for(n_ref);
    k_nn_init<<<1, 1, 0, s>>>(L.hdr);
    k_nn_bounds<<<blocks_for(n_ref + n_q), 256, 0, s>>>(ref, n_ref, q, n_q, L.hdr);
    k_nn_setup<<<1, 1, 0, s>>>(L.hdr, budget);
    cudaMemsetAsync(L.cnt, 0, (budget + 1) * 4, s);
    cudaMemsetAsync(L.bcnt, 0, (budget / kBlock + 2) * 4, s);
    if (n_ref > 0) k_nn_count<<<blocks_for(n_ref), 256, 0, s>>>(ref, n_ref, L.hdr, L.cnt, L.bcnt);
    // offsets over the whole budget (cells past ncell stay empty)
    launch_exclusive_scan(L.cnt, (long long)budget + 1, L.off, L.tile, &L.hdr->total, s);
    cudaMemsetAsync(L.cnt, 0, (budget + 1) * 4, s);
    if (n_ref > 0)
        k_nn_scatter<<<blocks_for(n_ref), 256, 0, s>>>(ref, n_ref, L.hdr, L.off, L.cnt, L.pts);
    k_nn_query<<<blocks_for(n_q), 256, 0, s>>>(q, n_q, L.hdr, L.off, L.bcnt, L.pts, dist);
}

size_t quality_partials_bytes() { return up256(sizeof(RedPart) * kRedBlocks) + 256; }

void launch_quality_reduce(const float *d_pred, long long n_pred, const float *d_gt,
                           long long n_gt, float tol, void *partials, double *out6,
                           cudaStream_t s) {
    RedPart *part = static_cast<RedPart *>(partials);
    k_quality_partials<<<kRedBlocks, kRedThreads, 0, s>>>(d_pred, n_pred, d_gt, n_gt, tol, part);
    k_quality_final<<<1, 1, 0, s>>>(part, n_pred, n_gt, out6);
}

void launch_centroids(const float *tri, long long n, float *out, cudaStream_t s) {
    if (n > 0) k_centroids<<<blocks_for(n), 256, 0, s>>>(tri, n, out);
}

}  // namespace dbt
