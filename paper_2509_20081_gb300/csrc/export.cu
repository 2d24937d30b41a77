// Map export: the signed-distance field and a triangle mesh of its
// iso-surface by Marching Cubes (Sec. III-C, Fig. 3: the map is exported as
// a Marching Cubes mesh at iso = 0).
//
// Field: sdf(v) = (sign ? +1 : -1) * popcount(mask) * res at the voxel
// centres (the distance is the number of set bits, Sec. III-A; the sign flag
// says free or occupied, Eq. 6).
//
// Mesh: a cell is the cube between 2 x 2 x 2 neighbouring voxel centres,
// corner q at (+x if bit 0, +y if bit 1, +z if bit 2); a corner is inside
// when sdf < iso.  The vertex on a crossed edge from lower corner a to upper
// corner b sits at t = (iso - f_a) / (f_b - f_a) along the edge, evaluated in
// binary64 with round-to-nearest intrinsics and rounded to float once.
// Triangles are listed by cell, x fastest over the box, then in table order,
// so the output is deterministic.
//
// The configuration table is derived at compile time from the cube itself:
// on each face the boundary is walked counter-clockwise as seen from outside,
// and each stretch of inside corners is closed by a segment from the crossing
// where the walk leaves it back to the crossing where it entered (so two
// diagonal inside corners of a face stay apart, on both cells sharing the
// face: the surface is closed).  The segments chain into loops, each
// started at its lowest edge and fanned from its first vertex whose
// diagonals never join two edges of one face (such a diagonal would lie in
// the face, on the neighbouring cell's surface); with that apex as e_0 the
// loop (e_0 .. e_m-1) gives (e_0, e_i+1, e_i), right-hand normal to sdf > iso.
#include "dbt_internal.cuh"

namespace dbt {

// ------------------------------------------------------------------ table
// Edge e = 4 * axis + j joins lower corner mc_edge_lo(e) to that corner plus
// the axis bit; j counts the four parallel edges by the other two coordinates.
__host__ __device__ constexpr int mc_edge_lo(int e) {
    const int axis = e >> 2, j = e & 3;
    return axis == 0 ? ((j & 1) << 1) | ((j >> 1) << 2)
         : axis == 1 ? (j & 1) | ((j >> 1) << 2)
                     : j;
}

constexpr int mc_edge_between(int a, int b) {
    const int d = a ^ b;
    const int axis = d == 1 ? 0 : d == 2 ? 1 : 2;
    const int lo = a < b ? a : b;
    const int j = axis == 0 ? ((lo >> 1) & 1) | (((lo >> 2) & 1) << 1)
                : axis == 1 ? (lo & 1) | (((lo >> 2) & 1) << 1)
                            : lo;
    return 4 * axis + j;
}

// Corner k of face (axis, side), counter-clockwise seen from outside: with
// (u, v) the next two axes in cyclic order, (0,0) (1,0) (1,1) (0,1) turns
// about +axis, so the + face uses it and the - face runs it backwards.
constexpr int mc_face_corner(int axis, int side, int k) {
    constexpr int cu[4] = {0, 1, 1, 0}, cv[4] = {0, 0, 1, 1};
    const int kk = side ? k : (4 - k) & 3;
    const int u = (axis + 1) % 3, v = (axis + 2) % 3;
    return (side << axis) | (cu[kk] << u) | (cv[kk] << v);
}

// Edges e and f lie on one face: some axis fixes the same coordinate on both.
constexpr bool mc_share_face(int e, int f) {
    const int ae = e >> 2, af = f >> 2;
    const int le = mc_edge_lo(e), lf = mc_edge_lo(f);
    for (int a = 0; a < 3; ++a) {
        if (a == ae || a == af) continue;          // the edge runs along a
        if (((le >> a) & 1) == ((lf >> a) & 1)) return true;
    }
    return false;
}

constexpr int MC_MAX_TRI = 5;

struct alignas(16) McTable {
    uint8_t ntri[256];
    uint8_t edge[256][3 * MC_MAX_TRI];
};

constexpr McTable build_mc_table() {
    McTable t{};
    for (int cfg = 0; cfg < 256; ++cfg) {
        int next[12] = {-1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1};
        for (int f = 0; f < 6; ++f) {
            const int axis = f >> 1, side = f & 1;
            bool in[4] = {};
            int side_edge[4] = {};
            for (int k = 0; k < 4; ++k) {
                in[k] = (cfg >> mc_face_corner(axis, side, k)) & 1;
                side_edge[k] = mc_edge_between(mc_face_corner(axis, side, k),
                                               mc_face_corner(axis, side, (k + 1) & 3));
            }
            for (int k = 0; k < 4; ++k) {
                if (!in[k] || in[(k + 1) & 3]) continue;          // side k does not leave
                int j = (k + 3) & 3;
                while (!( !in[j] && in[(j + 1) & 3])) j = (j + 3) & 3;   // entering side before it
                next[side_edge[k]] = side_edge[j];
            }
        }
        bool seen[12] = {};
        int n = 0;
        for (int e0 = 0; e0 < 12; ++e0) {
            if (next[e0] < 0 || seen[e0]) continue;
            int loop[12] = {};
            int m = 0;
            for (int e = e0; !seen[e]; e = next[e]) {
                seen[e] = true;
                loop[m++] = e;
            }
            int apex = 0;
            for (int a = m - 1; a >= 0; --a) {
                bool ok = true;
                for (int k = 2; k + 1 < m; ++k) ok = ok && !mc_share_face(loop[a], loop[(a + k) % m]);
                if (ok) apex = a;
            }
            for (int i = 1; i + 1 < m; ++i) {
                t.edge[cfg][3 * n + 0] = (uint8_t)loop[apex];
                t.edge[cfg][3 * n + 1] = (uint8_t)loop[(apex + i + 1) % m];
                t.edge[cfg][3 * n + 2] = (uint8_t)loop[(apex + i) % m];
                ++n;
            }
        }
        t.ntri[cfg] = (uint8_t)n;
    }
    return t;
}

constexpr McTable kMcTable = build_mc_table();
static_assert(kMcTable.ntri[0] == 0 && kMcTable.ntri[255] == 0 && kMcTable.ntri[1] == 1,
              "marching cubes table");

__device__ const McTable g_mc = kMcTable;

// ------------------------------------------------------------------ field
__device__ __forceinline__ double voxel_sdf(const DevGrid &g, size_t v, double res) {
    const double s = __ldg(g.sign + v) ? 1.0 : -1.0;
    return __dmul_rn(__dmul_rn(s, (double)__popc(__ldg(g.mask + v))), res);
}

__global__ void __launch_bounds__(256) k_sdf_field(DevGrid g, double res, ExportBox b,
                                                   float *__restrict__ out) {
    const long long n = (long long)b.bx * b.by * b.bz;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const long long x = i % b.bx, yz = i / b.bx;
        const long long y = yz % b.by, z = yz / b.by;
        const size_t v = ((size_t)(b.z0 + z) * g.ny + (size_t)(b.y0 + y)) * g.pitch +
                         (size_t)(b.x0 + x);
        out[i] = (float)voxel_sdf(g, v, res);
    }
}

// ------------------------------------------------------------------ cells
// A warp walks one unit of MC_UNIT consecutive cells, 32 per step.
constexpr int MC_UNIT = 1024;
constexpr int MC_STEPS = MC_UNIT / 32;

struct CellWalk {
    long long i, j, k;      // cell coordinates inside the box
};

__device__ __forceinline__ CellWalk cell_at(const ExportBox &b, long long L) {
    CellWalk c;
    c.i = L % b.cx;
    const long long r = L / b.cx;
    c.j = r % b.cy;
    c.k = r / b.cy;
    return c;
}

__device__ __forceinline__ void cell_advance(const ExportBox &b, CellWalk &c, int d) {
    c.i += d;
    while (c.i >= b.cx) {
        c.i -= b.cx;
        if (++c.j == b.cy) {
            c.j = 0;
            ++c.k;
        }
    }
}

__device__ __forceinline__ size_t cell_base(const DevGrid &g, const ExportBox &b, const CellWalk &c) {
    return ((size_t)(b.z0 + c.k) * g.ny + (size_t)(b.y0 + c.j)) * g.pitch + (size_t)(b.x0 + c.i);
}

// Inside bit of a voxel from the host-built table over (sign, popcount):
// bit s * 33 + p of lut says (s ? p : -p) * res < iso.
__device__ __forceinline__ uint32_t voxel_inside(const DevGrid &g, size_t v, uint64_t lut0,
                                                 uint64_t lut1) {
    const int idx = (__ldg(g.sign + v) ? 33 : 0) + __popc(__ldg(g.mask + v));
    return (uint32_t)(((idx < 64 ? lut0 >> idx : lut1 >> (idx - 64))) & 1ull);
}

__device__ __forceinline__ int cell_config(const DevGrid &g, size_t v0, uint64_t lut0, uint64_t lut1) {
    const size_t sy = (size_t)g.pitch, sz = (size_t)g.pitch * g.ny;
    int cfg = 0;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        const size_t v = v0 + ((q & 1) ? 1 : 0) + ((q & 2) ? sy : 0) + ((q & 4) ? sz : 0);
        cfg |= (int)voxel_inside(g, v, lut0, lut1) << q;
    }
    return cfg;
}

__global__ void __launch_bounds__(256) k_mc_count(DevGrid g, ExportBox b, uint64_t lut0,
                                                  uint64_t lut1, long long n_units,
                                                  uint32_t *__restrict__ unit_count) {
    __shared__ uint8_t s_ntri[256];
    for (int c = threadIdx.x; c < 256; c += blockDim.x) s_ntri[c] = g_mc.ntri[c];
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const long long warps = (long long)gridDim.x * (blockDim.x >> 5);
    for (long long u = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); u < n_units;
         u += warps) {
        const long long L0 = u * MC_UNIT + lane;
        CellWalk c = cell_at(b, L0 < b.ncell ? L0 : 0);
        uint32_t total = 0;
        for (int s = 0; s < MC_STEPS; ++s) {
            const long long L = L0 + 32LL * s;
            uint32_t nt = 0;
            if (L < b.ncell) nt = s_ntri[cell_config(g, cell_base(g, b, c), lut0, lut1)];
            total += __reduce_add_sync(0xffffffffu, nt);
            if (L + 32 < b.ncell) cell_advance(b, c, 32);
        }
        if (lane == 0) unit_count[u] = total;
    }
}

// ------------------------------------------------------------------ scan
constexpr int SCAN_THREADS = 1024;

// Exclusive prefix of v over the CTA (x-order of threads); *total gets the sum.
__device__ __forceinline__ unsigned long long cta_exclusive(unsigned long long v,
                                                            unsigned long long *total) {
    __shared__ unsigned long long s_w[SCAN_THREADS / 32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    unsigned long long x = v;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const unsigned long long y = __shfl_up_sync(0xffffffffu, x, d);
        if (lane >= d) x += y;
    }
    if (lane == 31) s_w[w] = x;
    __syncthreads();
    if (w == 0) {
        const int nw = blockDim.x >> 5;
        unsigned long long t = lane < nw ? s_w[lane] : 0ull;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const unsigned long long y = __shfl_up_sync(0xffffffffu, t, d);
            if (lane >= d) t += y;
        }
        if (lane < nw) s_w[lane] = t;
    }
    __syncthreads();
    const unsigned long long before = w ? s_w[w - 1] : 0ull;
    *total = s_w[(blockDim.x >> 5) - 1];
    __syncthreads();
    return before + x - v;
}

// Pass A: the sum of each CTA's tile of SCAN_THREADS units.
__global__ void __launch_bounds__(SCAN_THREADS) k_mc_scan_tiles(const uint32_t *__restrict__ cnt,
                                                                long long n,
                                                                unsigned long long *tile_sum) {
    const long long u = (long long)blockIdx.x * SCAN_THREADS + threadIdx.x;
    unsigned long long tot;
    cta_exclusive(u < n ? cnt[u] : 0u, &tot);
    if (threadIdx.x == 0) tile_sum[blockIdx.x] = tot;
}

// Pass B (one CTA): tile sums -> exclusive tile offsets; the grand total.
__global__ void __launch_bounds__(SCAN_THREADS) k_mc_scan_sums(unsigned long long *tile_sum,
                                                               long long n_tiles,
                                                               unsigned long long *total) {
    unsigned long long base = 0;
    for (long long t0 = 0; t0 < n_tiles; t0 += SCAN_THREADS) {
        const long long t = t0 + threadIdx.x;
        const unsigned long long v = t < n_tiles ? tile_sum[t] : 0ull;
        unsigned long long tot;
        const unsigned long long ex = cta_exclusive(v, &tot);
        if (t < n_tiles) tile_sum[t] = base + ex;
        base += tot;
    }
    if (threadIdx.x == 0) *total = base;
}

// Pass C: unit offsets = tile offset + exclusive prefix inside the tile.
__global__ void __launch_bounds__(SCAN_THREADS) k_mc_scan_units(const uint32_t *__restrict__ cnt,
                                                                long long n,
                                                                const unsigned long long *tile_off,
                                                                unsigned long long *unit_off) {
    const long long u = (long long)blockIdx.x * SCAN_THREADS + threadIdx.x;
    unsigned long long tot;
    const unsigned long long ex = cta_exclusive(u < n ? cnt[u] : 0u, &tot);
    if (u < n) unit_off[u] = tile_off[blockIdx.x] + ex;
}

// ------------------------------------------------------------------ emit
__global__ void __launch_bounds__(256) k_mc_emit(DevGrid g, ExportBox b, double res, double iso,
                                                 uint64_t lut0, uint64_t lut1, long long n_units,
                                                 const unsigned long long *__restrict__ unit_off,
                                                 float *__restrict__ tri, long long *__restrict__ cell,
                                                 long long max_tri) {
    __shared__ McTable s_mc;
    {
        const uint32_t *src = reinterpret_cast<const uint32_t *>(&g_mc);
        uint32_t *dst = reinterpret_cast<uint32_t *>(&s_mc);
        for (int c = threadIdx.x; c < (int)(sizeof(McTable) / 4); c += blockDim.x) dst[c] = src[c];
    }
    __syncthreads();
    const double org[3] = {g.ox, g.oy, g.oz};
    const size_t sy = (size_t)g.pitch, sz = (size_t)g.pitch * g.ny;
    const int lane = threadIdx.x & 31;
    const long long warps = (long long)gridDim.x * (blockDim.x >> 5);
    for (long long u = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); u < n_units;
         u += warps) {
        const long long L0 = u * MC_UNIT + lane;
        CellWalk c = cell_at(b, L0 < b.ncell ? L0 : 0);
        unsigned long long off = unit_off[u];
        for (int s = 0; s < MC_STEPS; ++s) {
            const long long L = L0 + 32LL * s;
            int cfg = 0, nt = 0;
            size_t v0 = 0;
            if (L < b.ncell) {
                v0 = cell_base(g, b, c);
                cfg = cell_config(g, v0, lut0, lut1);
                nt = s_mc.ntri[cfg];
            }
            int incl = nt;
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, incl, d);
                if (lane >= d) incl += y;
            }
            const int step_total = __shfl_sync(0xffffffffu, incl, 31);
            if (nt) {
                const long long base[3] = {b.x0 + c.i, b.y0 + c.j, b.z0 + c.k};
                for (int t = 0; t < nt; ++t) {
                    const unsigned long long id = off + (unsigned long long)(incl - nt + t);
                    if (id >= (unsigned long long)max_tri) break;
                    float *o = tri + 9ull * id;
#pragma unroll
                    for (int k = 0; k < 3; ++k) {
                        const int e = s_mc.edge[cfg][3 * t + k];
                        const int axis = e >> 2;
                        const int a = mc_edge_lo(e), bq = a | (1 << axis);
                        const size_t va = v0 + ((a & 1) ? 1 : 0) + ((a & 2) ? sy : 0) + ((a & 4) ? sz : 0);
                        const size_t vb = v0 + ((bq & 1) ? 1 : 0) + ((bq & 2) ? sy : 0) + ((bq & 4) ? sz : 0);
                        const double fa = voxel_sdf(g, va, res), fb = voxel_sdf(g, vb, res);
                        const double tt = __ddiv_rn(__dsub_rn(iso, fa), __dsub_rn(fb, fa));
#pragma unroll
                        for (int d = 0; d < 3; ++d) {
                            double q = __dadd_rn((double)(base[d] + ((a >> d) & 1)), 0.5);
                            if (d == axis) q = __dadd_rn(q, tt);
                            o[3 * k + d] = __double2float_rn(__dadd_rn(org[d], __dmul_rn(res, q)));
                        }
                    }
                    if (cell) cell[id] = L;
                }
            }
            off += (unsigned long long)step_total;
            if (L + 32 < b.ncell) cell_advance(b, c, 32);
        }
    }
}

// ------------------------------------------------------------------ launchers
long long mc_units(const ExportBox &b) { return (b.ncell + MC_UNIT - 1) / MC_UNIT; }

size_t mc_scratch_bytes(const ExportBox &b) {
    const long long nu = mc_units(b);
    const long long nt = (nu + SCAN_THREADS - 1) / SCAN_THREADS;
    auto up = [](size_t x) { return (x + 255) & ~size_t(255); };
    return up(256) + up((size_t)nu * 4) + up((size_t)nu * 8) + up((size_t)nt * 8);
}

static void mc_layout(const ExportBox &b, void *scratch, unsigned long long **total,
                      uint32_t **cnt, unsigned long long **uoff, unsigned long long **toff) {
    const long long nu = mc_units(b);
    auto up = [](size_t x) { return (x + 255) & ~size_t(255); };
    char *p = static_cast<char *>(scratch);
    *total = reinterpret_cast<unsigned long long *>(p);
    p += up(256);
    *cnt = reinterpret_cast<uint32_t *>(p);
    p += up((size_t)nu * 4);
    *uoff = reinterpret_cast<unsigned long long *>(p);
    p += up((size_t)nu * 8);
    *toff = reinterpret_cast<unsigned long long *>(p);
}

static int grid_for(long long work, int per_block) {
    const long long b = (work + per_block - 1) / per_block;
    return (int)std::max(1LL, std::min(b, (long long)152 * 16));
}

void launch_sdf_field(const DevGrid &g, double res, const ExportBox &b, float *out, cudaStream_t s) {
    const long long n = (long long)b.bx * b.by * b.bz;
    if (n > 0) k_sdf_field<<<grid_for(n, 256), 256, 0, s>>>(g, res, b, out);
}

void launch_mc_count(const DevGrid &g, const ExportBox &b, uint64_t lut0, uint64_t lut1,
                     void *scratch, cudaStream_t s) {
    unsigned long long *total, *uoff, *toff;
    uint32_t *cnt;
    mc_layout(b, scratch, &total, &cnt, &uoff, &toff);
    const long long nu = mc_units(b);
    if (nu == 0) {
        cudaMemsetAsync(total, 0, sizeof(unsigned long long), s);
        return;
    }
    const long long nt = (nu + SCAN_THREADS - 1) / SCAN_THREADS;
    k_mc_count<<<grid_for(nu, 8), 256, 0, s>>>(g, b, lut0, lut1, nu, cnt);
    k_mc_scan_tiles<<<(unsigned)nt, SCAN_THREADS, 0, s>>>(cnt, nu, toff);
    k_mc_scan_sums<<<1, SCAN_THREADS, 0, s>>>(toff, nt, total);
    k_mc_scan_units<<<(unsigned)nt, SCAN_THREADS, 0, s>>>(cnt, nu, toff, uoff);
}

void launch_mc_emit(const DevGrid &g, const ExportBox &b, double res, double iso, uint64_t lut0,
                    uint64_t lut1, void *scratch, float *tri, long long *cell, long long max_tri,
                    cudaStream_t s) {
    unsigned long long *total, *uoff, *toff;
    uint32_t *cnt;
    mc_layout(b, scratch, &total, &cnt, &uoff, &toff);
    const long long nu = mc_units(b);
    if (nu == 0 || max_tri <= 0) return;
    k_mc_emit<<<grid_for(nu, 8), 256, 0, s>>>(g, b, res, iso, lut0, lut1, nu, uoff, tri, cell,
                                              max_tri);
}

const unsigned long long *mc_total_ptr(void *scratch) {
    return static_cast<const unsigned long long *>(scratch);
}

void mc_table_host(uint8_t *ntri, uint8_t *edges) {
    for (int c = 0; c < 256; ++c) {
        ntri[c] = kMcTable.ntri[c];
        for (int k = 0; k < 3 * MC_MAX_TRI; ++k) edges[3 * MC_MAX_TRI * c + k] = kMcTable.edge[c][k];
    }
}

}  // namespace dbt
