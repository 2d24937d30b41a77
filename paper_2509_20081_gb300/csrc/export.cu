// Map export: the signed-distance field and a triangle mesh of its
// iso-surface by Marching Cubes (Sec. III-C, Fig. 3: the map is exported as
// a Marching Cubes mesh at iso = 0).
//
// Field: sdf(v) = (sign ? +1 : -1) * popcount(mask) * res at the voxel
// centres (the distance is the number of set bits, Sec. III-A; the sign flag
// says free or occupied, Eq. 6).
//
// Mesh: the field at a voxel centre is f = (sign ? +1 : -1) * popcount *
// res in binary32 (res and iso rounded to float once); a cell is the cube
// between 2 x 2 x 2 neighbouring voxel centres, corner q at (+x if bit 0, +y
// if bit 1, +z if bit 2); a corner is inside when f < iso.  The vertex on a
// crossed edge from lower corner a to upper corner b sits at
// t = (iso - f_a) / (f_b - f_a) along the edge, coordinate origin + res *
// ((index + 0.5) + t), every step a binary32 round-to-nearest intrinsic (the
// mesh is a float mesh; binary64 would run on the slow FP64 pipe).
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

// q = a / d, r = a % d for a >= 0, d > 0; 32-bit division when both fit
// (64-bit division is a long software sequence).
__device__ __forceinline__ void divmod(long long a, long long d, long long &q, long long &r) {
    if (((unsigned long long)a | (unsigned long long)d) >> 32) {
        q = a / d;
    } else {
        q = (long long)((uint32_t)a / (uint32_t)d);
    }
    r = a - q * d;
}

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
        long long x, yz, y, z;
        divmod(i, b.bx, yz, x);
        divmod(yz, b.by, z, y);
        const size_t v = ((size_t)(b.z0 + z) * g.ny + (size_t)(b.y0 + y)) * g.pitch +
                         (size_t)(b.x0 + x);
        out[i] = (float)voxel_sdf(g, v, res);
    }
}

// ------------------------------------------------------------------ cells
// Pass 0 turns the box into an inside bit plane: bit x of word
// ((z * by + y) * wpr + x / 32) is voxel (x0 + x, y0 + y, z0 + z) < iso.
//
// The cells are then walked in units: a unit is a segment of up to 1024
// consecutive cells of one cell row (fixed j, k), so units are contiguous
// and ordered in the cell numbering L; a warp takes a unit and lane l the
// 32 cells x = 1024 u + 32 l .. + 31, whose 2 x 2 x 2 corner bits come from
// four 33-bit windows of the plane (rows j, j+1 of slices k, k+1).  A cell
// with all eight bits equal has no triangle, so a lane visits only the set
// bits of its "mixed" mask: the work follows the surface, not the volume.
constexpr int MC_LEVELS = 66;          // (sign, popcount) pairs: s * 33 + p
constexpr int MC_SEG = 1024;           // cells per unit

__device__ __forceinline__ size_t voxel_index(const DevGrid &g, const ExportBox &b, long long x,
                                              long long y, long long z) {
    return ((size_t)(b.z0 + z) * g.ny + (size_t)(b.y0 + y)) * g.pitch + (size_t)(b.x0 + x);
}

__device__ __forceinline__ int voxel_level(const DevGrid &g, size_t v) {
    return (__ldg(g.sign + v) ? 33 : 0) + __popc(__ldg(g.mask + v));
}

// Inside test of a voxel: f = (s ? +1 : -1) * p * res is monotone in p for
// each sign, so f < iso is p < p_free for free voxels and p > p_occ for
// occupied ones (thresholds derived on the host from the same comparison).
__device__ __forceinline__ bool inside_of(uint32_t mask, uint32_t sign, int p_free, int p_occ) {
    const int pc = __popc(mask);
    return sign ? pc < p_free : pc > p_occ;
}

// One warp per plane row.  With x0 a multiple of 4 (rows 16-byte aligned)
// each lane reads four voxels at once (uint4 masks, one word of signs) into
// a 4-bit nibble, and eight lanes' nibbles OR-reduce (three xor shuffles)
// into one word of 32 voxels; otherwise one voxel per lane per word.
__global__ void __launch_bounds__(256) k_mc_bits(DevGrid g, ExportBox b, int p_free, int p_occ,
                                                 int wpr, uint32_t *__restrict__ bits) {
    const int lane = threadIdx.x & 31;
    const long long rows = (long long)b.by * b.bz;
    const long long warps = (long long)gridDim.x * (blockDim.x >> 5);
    const bool vec = (b.x0 & 3) == 0;
    for (long long r = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); r < rows;
         r += warps) {
        long long y, z;
        divmod(r, b.by, z, y);
        const size_t v0 = voxel_index(g, b, 0, y, z);
        const uint32_t *mrow = g.mask + v0;
        const uint8_t *srow = g.sign + v0;
        uint32_t *out = bits + r * wpr;
        if (vec) {
            for (int x0 = 0; x0 < b.bx; x0 += 256) {        // two chunks of 128 in flight
                uint32_t nib[2] = {0u, 0u};                   // bit q: voxel 4 lane + q inside
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int x = x0 + 128 * h + 4 * lane;
                    if (x + 3 < b.bx) {
                        const uint4 m4 = __ldg(reinterpret_cast<const uint4 *>(mrow + x));
                        const uint32_t s4 = __ldg(reinterpret_cast<const uint32_t *>(srow + x));
                        nib[h] = (uint32_t)inside_of(m4.x, s4 & 0xFFu, p_free, p_occ) |
                                 ((uint32_t)inside_of(m4.y, (s4 >> 8) & 0xFFu, p_free, p_occ) << 1) |
                                 ((uint32_t)inside_of(m4.z, (s4 >> 16) & 0xFFu, p_free, p_occ) << 2) |
                                 ((uint32_t)inside_of(m4.w, s4 >> 24, p_free, p_occ) << 3);
                    } else {
#pragma unroll
                        for (int q = 0; q < 4; ++q)
                            if (x + q < b.bx &&
                                inside_of(__ldg(mrow + x + q), __ldg(srow + x + q), p_free, p_occ))
                                nib[h] |= 1u << q;
                    }
                }
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    // eight lanes' nibbles form one 32-voxel word (lane l at bits 4 (l & 7))
                    uint32_t v = nib[h] << (4 * (lane & 7));
                    v |= __shfl_xor_sync(0xffffffffu, v, 1);
                    v |= __shfl_xor_sync(0xffffffffu, v, 2);
                    v |= __shfl_xor_sync(0xffffffffu, v, 4);
                    const int w = ((x0 + 128 * h) >> 5) + (lane >> 3);
                    if ((lane & 7) == 0 && w < wpr) out[w] = v;
                }
            }
        } else {
            for (int w0 = 0; w0 < wpr; w0 += 4) {
                bool in[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) {         // four words' loads in flight
                    const int x = 32 * (w0 + q) + lane;
                    in[q] = x < b.bx && inside_of(__ldg(mrow + x), __ldg(srow + x), p_free, p_occ);
                }
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const uint32_t word = __ballot_sync(0xffffffffu, in[q]);
                    if (lane == 0 && w0 + q < wpr) out[w0 + q] = word;
                }
            }
        }
    }
}

struct Unit {
    long long j, k;         // cell row
    long long x0;           // first cell of the unit in the row
};

__device__ __forceinline__ Unit unit_at(const ExportBox &b, long long upr, long long u) {
    Unit t;
    long long row, seg;
    divmod(u, upr, row, seg);
    t.x0 = seg * MC_SEG;
    divmod(row, b.cy, t.k, t.j);
    return t;
}

// The lane's 32 cells from x = xs: its four windows (bit s and s + 1 of each
// for cell xs + s), and the mask of cells that exist and are mixed.
struct LaneCells {
    uint64_t w00, w10, w01, w11;   // rows (j, k), (j+1, k), (j, k+1), (j+1, k+1)
    uint32_t mixed;
};

__device__ __forceinline__ uint64_t window(const uint32_t *bits, int wpr, long long row, long long w) {
    const uint32_t *p = bits + row * wpr;
    const uint64_t lo = w < wpr ? __ldg(p + w) : 0u;
    const uint64_t hi = w + 1 < wpr ? (__ldg(p + w + 1) & 1u) : 0u;
    return lo | (hi << 32);
}

__device__ __forceinline__ LaneCells lane_cells(const uint32_t *bits, int wpr, const ExportBox &b,
                                                const Unit &t, int lane) {
    LaneCells c;
    const long long xs = t.x0 + 32LL * lane;
    const long long w = xs >> 5;
    const long long r = t.k * b.by + t.j;
    c.w00 = window(bits, wpr, r, w);
    c.w10 = window(bits, wpr, r + 1, w);
    c.w01 = window(bits, wpr, r + b.by, w);
    c.w11 = window(bits, wpr, r + b.by + 1, w);
    const uint64_t o = c.w00 | c.w10 | c.w01 | c.w11, a = c.w00 & c.w10 & c.w01 & c.w11;
    const uint64_t o2 = o | (o >> 1), a2 = a & (a >> 1);   // bit s: cells s, s + 1 together
    const long long n = b.cx - xs;                        // cells of this lane that exist
    const uint32_t valid = n >= 32 ? 0xffffffffu : n <= 0 ? 0u : (1u << n) - 1u;
    c.mixed = (uint32_t)(o2 & ~a2) & valid;
    return c;
}

__device__ __forceinline__ int lane_config(const LaneCells &c, int s) {
    return (int)(((c.w00 >> s) & 3u) | (((c.w10 >> s) & 3u) << 2) | (((c.w01 >> s) & 3u) << 4) |
                 (((c.w11 >> s) & 3u) << 6));
}

__global__ void __launch_bounds__(256) k_mc_count(ExportBox b, const uint32_t *__restrict__ bits,
                                                  int wpr, long long upr, long long n_units,
                                                  uint32_t *__restrict__ unit_count) {
    __shared__ uint8_t s_ntri[256];
    for (int c = threadIdx.x; c < 256; c += blockDim.x) s_ntri[c] = g_mc.ntri[c];
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const long long warps = (long long)gridDim.x * (blockDim.x >> 5);
    for (long long u = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); u < n_units;
         u += warps) {
        const LaneCells c = lane_cells(bits, wpr, b, unit_at(b, upr, u), lane);
        uint32_t nt = 0;
        for (uint32_t m = c.mixed; m; m &= m - 1) nt += s_ntri[lane_config(c, __ffs(m) - 1)];
        nt = __reduce_add_sync(0xffffffffu, nt);
        if (lane == 0) unit_count[u] = nt;
    }
}

// Crossing fractions t = (iso - f_a) / (f_b - f_a) for every pair of levels
// (f = (s ? +1 : -1) * p * res), in binary32, once per call; entries of
// pairs on the same side of iso are never read.
__global__ void k_mc_fractions(float res, float iso, float *__restrict__ tab) {
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < MC_LEVELS * MC_LEVELS;
         e += gridDim.x * blockDim.x) {
        const int la = e / MC_LEVELS, lb = e % MC_LEVELS;
        const float fa = __fmul_rn(__fmul_rn(la >= 33 ? 1.0f : -1.0f, (float)(la % 33)), res);
        const float fb = __fmul_rn(__fmul_rn(lb >= 33 ? 1.0f : -1.0f, (float)(lb % 33)), res);
        tab[e] = fa == fb ? 0.0f : __fdiv_rn(__fsub_rn(iso, fa), __fsub_rn(fb, fa));
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
// Position of the n-th (0-based) set bit of m, n < popc(m).
__device__ __forceinline__ int nth_set_bit(uint32_t m, int n) {
    int pos = 0;
#pragma unroll
    for (int w = 16; w; w >>= 1) {
        const int c = __popc(m & ((1u << w) - 1u));
        if (n >= c) {
            n -= c;
            m >>= w;
            pos += w;
        }
    }
    return pos;
}

__device__ __forceinline__ uint64_t shfl64(uint64_t v, int src) {
    const uint32_t lo = __shfl_sync(0xffffffffu, (uint32_t)v, src);
    const uint32_t hi = __shfl_sync(0xffffffffu, (uint32_t)(v >> 32), src);
    return (uint64_t)lo | ((uint64_t)hi << 32);
}

// A warp takes a unit with triangles and deals its surface cells (the mixed
// bits of all lanes, in cell order) out 32 at a time, one per lane: lane l
// of a round gets the cell of rank 32 r + l, found from the lanes' prefix
// counts by a binary search over shuffles.
__device__ __forceinline__ float mc_coord(float org, float res, long long idx, float t) {
    return __fadd_rn(org, __fmul_rn(res, __fadd_rn(__fadd_rn(__ll2float_rn(idx), 0.5f), t)));
}

__global__ void __launch_bounds__(256, 4) k_mc_emit(DevGrid g, ExportBox b, float res,
                                                    const uint32_t *__restrict__ bits, int wpr,
                                                    long long upr, const float *__restrict__ frac,
                                                    long long n_units,
                                                    const unsigned long long *__restrict__ unit_off,
                                                    const uint32_t *__restrict__ unit_count,
                                                    float *__restrict__ tri,
                                                    long long *__restrict__ cell, long long max_tri) {
    __shared__ McTable s_mc;
    __shared__ float s_frac[MC_LEVELS * MC_LEVELS];
    {
        const uint32_t *src = reinterpret_cast<const uint32_t *>(&g_mc);
        uint32_t *dst = reinterpret_cast<uint32_t *>(&s_mc);
        for (int c = threadIdx.x; c < (int)(sizeof(McTable) / 4); c += blockDim.x) dst[c] = src[c];
        for (int c = threadIdx.x; c < MC_LEVELS * MC_LEVELS; c += blockDim.x) s_frac[c] = frac[c];
    }
    __syncthreads();
    const float org[3] = {__double2float_rn(g.ox), __double2float_rn(g.oy), __double2float_rn(g.oz)};
    const int lane = threadIdx.x & 31;
    const long long warps = (long long)gridDim.x * (blockDim.x >> 5);
    for (long long u = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); u < n_units;
         u += warps) {
        if (unit_count[u] == 0) continue;                    // warp-uniform
        const Unit t = unit_at(b, upr, u);
        const LaneCells c = lane_cells(bits, wpr, b, t, lane);
        const int nm = __popc(c.mixed);
        int ex = nm;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, ex, d);
            if (lane >= d) ex += y;
        }
        const int n_surf = __shfl_sync(0xffffffffu, ex, 31);
        ex -= nm;                                             // exclusive prefix
        unsigned long long off = unit_off[u];
        const long long Lrow = (t.k * b.cy + t.j) * b.cx;
        const long long jy = b.y0 + t.j, kz = b.z0 + t.k;
        const float py[2] = {mc_coord(org[1], res, jy, 0.0f), mc_coord(org[1], res, jy + 1, 0.0f)};
        const float pz[2] = {mc_coord(org[2], res, kz, 0.0f), mc_coord(org[2], res, kz + 1, 0.0f)};
        for (int r0 = 0; r0 < n_surf; r0 += 32) {
            const int k = r0 + lane;
            int owner = 0;                                    // last lane with ex <= k
#pragma unroll
            for (int step = 16; step; step >>= 1) {
                const int e = __shfl_sync(0xffffffffu, ex, owner + step);
                if (e <= k) owner += step;
            }
            const uint32_t om = __shfl_sync(0xffffffffu, c.mixed, owner);
            const int oe = __shfl_sync(0xffffffffu, ex, owner);
            LaneCells oc;
            oc.w00 = shfl64(c.w00, owner);
            oc.w10 = shfl64(c.w10, owner);
            oc.w01 = shfl64(c.w01, owner);
            oc.w11 = shfl64(c.w11, owner);
            const bool have = k < n_surf;
            const int s = have ? nth_set_bit(om, k - oe) : 0;
            const int cfg = lane_config(oc, s);
            const int nt = have ? s_mc.ntri[cfg] : 0;
            int incl = nt;
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, incl, d);
                if (lane >= d) incl += y;
            }
            unsigned long long id = off + (unsigned long long)(incl - nt);
            off += (unsigned long long)__shfl_sync(0xffffffffu, incl, 31);
            if (!have || id >= (unsigned long long)max_tri) continue;
            const long long i = t.x0 + 32LL * owner + s;
            int lv[8];
#pragma unroll
            for (int q = 0; q < 8; ++q)
                lv[q] = voxel_level(g, voxel_index(g, b, i + (q & 1), t.j + ((q >> 1) & 1),
                                                   t.k + ((q >> 2) & 1)));
            const long long ix = b.x0 + i;
            const float px[2] = {mc_coord(org[0], res, ix, 0.0f), mc_coord(org[0], res, ix + 1, 0.0f)};
            const long long q0[3] = {ix, jy, kz};
            for (int tt = 0; tt < nt && id < (unsigned long long)max_tri; ++tt, ++id) {
                float *o = tri + 9ull * id;
#pragma unroll
                for (int kk = 0; kk < 3; ++kk) {
                    const int e = s_mc.edge[cfg][3 * tt + kk];
                    const int axis = e >> 2;
                    const int a = mc_edge_lo(e), bq = a | (1 << axis);
                    const float onaxis = mc_coord(org[axis], res, q0[axis],
                                                  s_frac[lv[a] * MC_LEVELS + lv[bq]]);
                    o[3 * kk + 0] = axis == 0 ? onaxis : px[a & 1];
                    o[3 * kk + 1] = axis == 1 ? onaxis : py[(a >> 1) & 1];
                    o[3 * kk + 2] = axis == 2 ? onaxis : pz[(a >> 2) & 1];
                }
                if (cell) cell[id] = Lrow + i;
            }
        }
    }
}

// ------------------------------------------------------------------ launchers
static long long mc_upr(const ExportBox &b) { return (b.cx + MC_SEG - 1) / MC_SEG; }

long long mc_units(const ExportBox &b) { return b.ncell ? mc_upr(b) * b.cy * b.cz : 0; }

static int mc_wpr(const ExportBox &b) { return (b.bx + 31) / 32; }

static size_t up256(size_t x) { return (x + 255) & ~size_t(255); }

// Scratch: [total | fractions | unit counts | unit offsets | tile sums | bit plane]
struct McLayout {
    unsigned long long *total;
    float *frac;
    uint32_t *cnt;
    unsigned long long *uoff, *toff;
    uint32_t *bits;
    size_t bytes;
};

static McLayout mc_layout(const ExportBox &b, void *scratch) {
    const long long nu = mc_units(b);
    const long long nt = (nu + SCAN_THREADS - 1) / SCAN_THREADS;
    const size_t nbits = (size_t)mc_wpr(b) * (size_t)b.by * (size_t)b.bz;
    McLayout m{};
    char *p = static_cast<char *>(scratch);
    size_t o = 0;
    m.total = reinterpret_cast<unsigned long long *>(p + o);
    o += up256(256);
    m.frac = reinterpret_cast<float *>(p + o);
    o += up256(sizeof(float) * MC_LEVELS * MC_LEVELS);
    m.cnt = reinterpret_cast<uint32_t *>(p + o);
    o += up256((size_t)nu * 4);
    m.uoff = reinterpret_cast<unsigned long long *>(p + o);
    o += up256((size_t)nu * 8);
    m.toff = reinterpret_cast<unsigned long long *>(p + o);
    o += up256((size_t)nt * 8);
    m.bits = reinterpret_cast<uint32_t *>(p + o);
    o += up256(nbits * 4);
    m.bytes = o;
    return m;
}

size_t mc_scratch_bytes(const ExportBox &b) { return mc_layout(b, nullptr).bytes; }

static int grid_for(long long work, int per_block) {
    const long long b = (work + per_block - 1) / per_block;
    return (int)std::max(1LL, std::min(b, 16LL * device_sm_count()));
}

void launch_sdf_field(const DevGrid &g, double res, const ExportBox &b, float *out, cudaStream_t s) {
    const long long n = (long long)b.bx * b.by * b.bz;
    if (n > 0) k_sdf_field<<<grid_for(n, 256), 256, 0, s>>>(g, res, b, out);
}

void launch_mc_count(const DevGrid &g, const ExportBox &b, uint64_t lut0, uint64_t lut1,
                     void *scratch, cudaStream_t s) {
    const McLayout m = mc_layout(b, scratch);
    const long long nu = mc_units(b);
    if (nu == 0) {
        cudaMemsetAsync(m.total, 0, sizeof(unsigned long long), s);
        return;
    }
    const long long nt = (nu + SCAN_THREADS - 1) / SCAN_THREADS;
    const int wpr = mc_wpr(b);
    // the inside levels of each sign are a run of popcounts (f is monotone in
    // p): free voxels p < p_free, occupied ones p > p_occ
    auto inside = [&](int lv) { return ((lv < 64 ? lut0 >> lv : lut1 >> (lv - 64)) & 1ull) != 0; };
    int p_free = 0, p_occ = 32;
    while (p_free <= 32 && inside(33 + p_free)) ++p_free;
    while (p_occ >= 0 && inside(p_occ)) --p_occ;
    k_mc_bits<<<grid_for((long long)b.by * b.bz, 8), 256, 0, s>>>(g, b, p_free, p_occ, wpr, m.bits);
    k_mc_count<<<grid_for(nu, 8), 256, 0, s>>>(b, m.bits, wpr, mc_upr(b), nu, m.cnt);
    k_mc_scan_tiles<<<(unsigned)nt, SCAN_THREADS, 0, s>>>(m.cnt, nu, m.toff);
    k_mc_scan_sums<<<1, SCAN_THREADS, 0, s>>>(m.toff, nt, m.total);
    k_mc_scan_units<<<(unsigned)nt, SCAN_THREADS, 0, s>>>(m.cnt, nu, m.toff, m.uoff);
}

void launch_mc_emit(const DevGrid &g, const ExportBox &b, double res, double iso, uint64_t lut0,
                    uint64_t lut1, void *scratch, float *tri, long long *cell, long long max_tri,
                    cudaStream_t s) {
    (void)lut0;
    (void)lut1;
    const McLayout m = mc_layout(b, scratch);
    const long long nu = mc_units(b);
    if (nu == 0 || max_tri <= 0) return;
    const float resf = (float)res, isof = (float)iso;
    k_mc_fractions<<<(MC_LEVELS * MC_LEVELS + 255) / 256, 256, 0, s>>>(resf, isof, m.frac);
    const int emit_ctas = std::min(grid_for(nu, 8), 8 * device_sm_count());
    k_mc_emit<<<emit_ctas, 256, 0, s>>>(g, b, resf, m.bits, mc_wpr(b), mc_upr(b), m.frac, nu, m.uoff,
                                        m.cnt, tri, cell, max_tri);
}

// Exclusive prefix sums of n counts into out, the grand total into *total;
// tile holds ceil(n / 1024) partial sums.
void launch_exclusive_scan(const uint32_t *cnt, long long n, unsigned long long *out,
                           unsigned long long *tile, unsigned long long *total, cudaStream_t s) {
    if (n <= 0) {
        cudaMemsetAsync(total, 0, sizeof(unsigned long long), s);
        return;
    }
    const long long nt = (n + SCAN_THREADS - 1) / SCAN_THREADS;
    k_mc_scan_tiles<<<(unsigned)nt, SCAN_THREADS, 0, s>>>(cnt, n, tile);
    k_mc_scan_sums<<<1, SCAN_THREADS, 0, s>>>(tile, nt, total);
    k_mc_scan_units<<<(unsigned)nt, SCAN_THREADS, 0, s>>>(cnt, n, tile, out);
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
