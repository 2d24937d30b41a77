// Brick integration of one scan (Sec. III-C, Eqs. 4-6).
//
// Distance codes.  A mask of the form 2^k - 1 is stored as k = popcount; the
// Eq. 4 AND of two such masks is the mask of min(k).  Grid masks start all
// ones (Sec. III-A) and only ever meet Eq. 3 masks, so they keep this form
// (checked on load; a violation latches ERR_MASK_FORM).
//
// Per brick, the kernels of all its (return, brick) pairs are first folded
// among themselves: a warp area holds, per voxel, the minimum code of the
// kernels applied so far (8-bit codes, four voxels per 32-bit word, 32 =
// none), so the AND of four voxels is one byte-wise minimum and nothing is
// read from the grid before the kernels are applied.  The grid's masks are
// read once, at write-back, where each covered voxel takes min(old, kernel
// minimum) -- the same result as AND-ing the kernels into the mask one by
// one, because the AND of masks of the form 2^k - 1 is the minimum of codes,
// which is associative and commutative.
//
// Kernel rows.  For a row of the K^3 kernel at squared lateral offset
// q = oy^2 + oz^2 the codes along x are ceil(sqrt(ox^2 + q)).  The host builds
// P[q][s]: the four codes a 4-voxel word receives when its first voxel sits
// at ox = s - 3 - R (32, no change, outside the kernel).  A word update is a
// table load, an area-word load, a byte-wise min and a conditional store.
//
// Work split.  Persistent CTAs of WPC warps.  Bricks (32 x 8 x BZ voxels;
// BZ = 4, 8 or 16, one kernel instance per depth) with more than ws.heavy
// (return, brick) pairs ("heavy") are taken one per group of warps: at
// K <= 13 by the separable dense path below, otherwise each warp applies a
// share of the pairs to its own area and the areas are merged at write-back
// (byte-wise min of codes, sum of counts).  The other bricks are taken one
// per warp, in size classes, largest first.  At K <= 11 (K <= 7 for BZ = 4)
// a CTA holds two groups of four warps, one starting on heavy and one on
// light bricks; otherwise the CTA is one group, heavy bricks first.  A brick
// is only ever written by the group or warp that took it, so no atomics
// touch the grid.
//
// Per brick:
//   I. the area cleared: no code (32) and zero counts,
//   C. every pair applied (lanes = the kernel rows inside the brick, each
//      updating the up to NW words of its row), then the bin's shadow offsets
//      that fall in the brick counted (Eq. 5),
//   D. write-back: every chunk of four voxels that some kernel covers reads
//      its masks, takes the minimum with the kernel codes and stores the
//      masks that change; chunks with shadow counts c take
//      h' = min(h + c, H_max) and sign 0 when h < T <= h' (Eq. 6).
// The saturating count with a threshold crossing depends only on the total
// count, so D gives exactly the state of applying the returns one by one in
// scan order (the first-return rule is resolved before this kernel).
#include <mutex>

#include "dbt_internal.cuh"

namespace dbt {

constexpr int WPC = 8;            // warps per CTA
constexpr int NTHR = WPC * 32;

// Rows of BX voxels (row = z * BY + y), chunks of four voxels and voxels of
// a brick of depth BZ.
template <int BZ> __host__ __device__ constexpr int brows() { return BY * BZ; }
template <int BZ> __host__ __device__ constexpr int bchunks() { return BY * BZ * CHUNKS_PER_ROW; }
template <int BZ> __host__ __device__ constexpr int bvox() { return BX * BY * BZ; }

template <int BZ>
struct WarpArea {
    uint32_t kst[brows<BZ>() * 8];  // kernel codes: word kword(row, w) = voxels 4w .. 4w+3 of a row
    uint16_t cnt[bvox<BZ>()];       // shadow counts, index row * 32 + x
};
static_assert(sizeof(WarpArea<4>) % 16 == 0 && sizeof(WarpArea<8>) % 16 == 0 &&
                  sizeof(WarpArea<16>) % 16 == 0, "warp area alignment");
constexpr uint32_t NO_CODE4 = 0x20202020u;      // four voxels without a kernel code (32)

// Word w of brick row `row` (row = z * BY + y).  The XOR with bits 2..4 of the
// row spreads both access patterns over all 32 banks: phase C (8 rows x 4
// consecutive planes, same w) and phase D (4 consecutive rows x 8 words).
__device__ __forceinline__ int kword(int row, int w) { return row * 8 + (w ^ ((row >> 2) & 7)); }

__device__ __forceinline__ uint32_t vmin4(uint32_t a, uint32_t b) { return __vminu4(a, b); }

// Named barrier `id` (1 + group index) over the n threads of a heavy-brick
// group of warps; id 0 is the whole CTA.
__device__ __forceinline__ void group_sync(int id, int n) {
    if (id == 0)
        __syncthreads();
    else if (id == 1)   // immediate barrier ids: the kernel then holds three barriers, not all 16
        asm volatile("bar.sync 1, %0;" ::"r"(n) : "memory");
    else
        asm volatile("bar.sync 2, %0;" ::"r"(n) : "memory");
}

// Bytes of b below the matching bytes of a, as bit 7 of each byte, for bytes
// < 128 (codes are <= 32): b + 128 - a per byte lies in [1, 255], so the
// subtraction never borrows across bytes and bit 7 is clear exactly when
// b < a.  code_min() then takes those bytes of b: the byte-wise minimum.
__device__ __forceinline__ uint32_t code_lt(uint32_t a, uint32_t b) {
    return ~((b | 0x80808080u) - a) & 0x80808080u;
}
__device__ __forceinline__ uint32_t code_min(uint32_t a, uint32_t b, uint32_t lt) {
    const uint32_t m = (lt >> 7) * 0xFFu;
    return (a & ~m) | (b & m);
}

__device__ __forceinline__ uint32_t code_to_mask(uint32_t k) {
    return k == 0u ? 0u : (0xFFFFFFFFu >> (32u - k));
}

struct PairBox {
    int cx, cy, cz;               // contact relative to the brick corner
    int x0, x1, y0, y1, z0, z1;   // kernel box clipped to the brick
};

template <int BZ>
__device__ __forceinline__ PairBox decode_pair(uint32_t pl, int R) {
    PairBox b;
    b.cx = (int)(pl & 63u) - R;
    b.cy = (int)((pl >> 6) & 31u) - R;
    b.cz = (int)((pl >> 11) & 31u) - R;
    b.x0 = max(b.cx - R, 0);
    b.x1 = min(b.cx + R, BX - 1);
    b.y0 = max(b.cy - R, 0);
    b.y1 = min(b.cy + R, BY - 1);
    b.z0 = max(b.cz - R, 0);
    b.z1 = min(b.cz + R, BZ - 1);
    return b;
}

// Phase C (Eq. 4) for one pair on a warp's area.  The box's wy x wz kernel
// rows are spread over the lanes (row r -> z = r / wy, y = r % wy, the
// division by wy <= 8 done exactly as (r * ceil(256 / wy)) >> 8 for r < 64);
// each lane lowers the codes of the up to NW words of its row.  Each lane
// owns its row within one pair, so no two lanes write one word.  The pair's
// set-up (clipped box, first word, table shift) is taken by the lane that
// holds the pair, for 32 pairs at once, and handed out packed in two words:
//   a = nrows | wy << 8 | y0 << 12 | z0 << 16 | nw << 21 | w0 << 24
//   b = s0 | (cy + 32) << 8 | (cz + 32) << 16
// The row split r / wy is (r * ceil(65536 / wy)) >> 16, exact for r < 1024.
struct RowsSetup {
    uint32_t a, b;
};

template <int BZ>
__device__ __forceinline__ RowsSetup rows_setup(uint32_t pl, int R) {
    const PairBox b = decode_pair<BZ>(pl, R);
    const int wy = b.y1 - b.y0 + 1;
    const int nrows = wy * (b.z1 - b.z0 + 1);
    const int w0 = b.x0 >> 2;
    const int nw = (b.x1 >> 2) - w0;
    const int s0 = 4 * w0 - b.cx + R + 3;
    RowsSetup su;
    su.a = (uint32_t)nrows | ((uint32_t)wy << 8) | ((uint32_t)b.y0 << 12) | ((uint32_t)b.z0 << 16) |
           ((uint32_t)nw << 21) | ((uint32_t)w0 << 24);
    su.b = (uint32_t)s0 | ((uint32_t)(b.cy + 32) << 8) | ((uint32_t)(b.cz + 32) << 16);
    return su;
}

template <int NW, int BZ>
__device__ __forceinline__ void apply_rows(RowsSetup su, WarpArea<BZ> *wa, const uint32_t *P, int W,
                                           int lane) {
    const int nrows = (int)(su.a & 255u);
    const int wy = (int)((su.a >> 8) & 15u);
    const int y0 = (int)((su.a >> 12) & 15u), z0 = (int)((su.a >> 16) & 31u);
    const int nw = (int)((su.a >> 21) & 7u), w0 = (int)((su.a >> 24) & 15u);
    // ceil(65536 / wy) - 1 for wy = 1..8 as 16-bit fields (no integer division)
    const uint64_t mt = wy <= 4 ? 0x3FFF55557FFFFFFFull : 0x1FFF24922AAA3333ull;
    const int magic = (int)((mt >> (16 * ((wy - 1) & 3))) & 0xFFFFull) + 1;
    const int s0 = (int)(su.b & 255u);
    const int cy = (int)((su.b >> 8) & 255u) - 32, cz = (int)((su.b >> 16) & 255u) - 32;
    for (int r = lane; r < nrows; r += 32) {
        const int qz = (r * magic) >> 16;
        const int ry = y0 + (r - qz * wy), rz = z0 + qz;
        const int oy = ry - cy, oz = rz - cz;
        const int pb = (oy * oy + oz * oz) * W + s0;
        const int row = rz * BY + ry;
        const int rbase = row * 8, f = (row >> 2) & 7;
#pragma unroll
        for (int j = 0; j < NW; ++j) {
            if (j <= nw) {
                const uint32_t kwd = P[pb + 4 * j];
                const int addr = rbase + ((w0 + j) ^ f);
                const uint32_t a = wa->kst[addr];
                const uint32_t lt = code_lt(a, kwd);
                if (lt) wa->kst[addr] = code_min(a, kwd, lt);
            }
        }
    }
}

// Eq. 5 counts of up to 32 pairs (lane j holds pair j's payload in `mine`,
// j < n): lanes walk each pair's shadow offsets and count those inside the
// brick.  The per-pair set-up is taken lane-parallel first: whether the
// contact lies within r_s of the brick (else no offset can fall in it), the
// contact packed as bytes, and the pair's range of offsets -- for a contact
// outside the brick along z only the offsets whose plane falls in the brick
// (a sub-range of the oz-major list, sh_zs), along y (z inside) only the
// rows that fall in it (oy-major list, sh_ys), else the bin's whole list.
// Then the pairs with offsets to walk are taken one by one (ballot).
// ATOMIC: several warps count into one array, so counts are added
// atomically to their packed 16-bit halves.  A pair adds at most 1 to a
// voxel, and a brick's pairs are counted in rounds of at most CNT_ROUND, so
// a count stays below 2^16; the write-back saturates the counter at H_max.
//
// Offsets are packed bytes o + 32 and the contact c relative to the brick
// is packed as bytes c + 32, so one 32-bit add gives per byte o + c + 64,
// which lies in [44, 115] (|o| <= SR <= 10, c in [-SR, 31 + SR]): no byte
// carries into the next.  The voxel o + c is in the brick exactly when that
// byte is in [64, 64 + BX) for x, [64, 64 + BY) for y and [64, 64 + BZ) for
// z, i.e. (for power-of-two sides dividing 64) when the bits above the side
// read 01: one AND and one compare.  Lanes past the range take 0x80 bytes,
// which set bit 7 and fail.  The low bits of the bytes are then x, y and z.
static_assert(BX == 32 && BY == 8 && MAX_R <= 10 && OFF_BIAS == 32 && BZ_MAX - 1 + 4 * MAX_R + 64 < 128,
              "shadow_pairs' byte packing: 32 x 8 x BZ bricks, |offsets| <= 10, no byte carry");
constexpr uint32_t SH_PAD = 0x80808080u;
template <int BZ>
__host__ __device__ constexpr uint32_t sh_inmask() {
    static_assert(BZ == 4 || BZ == 8 || BZ == 16, "brick depth");
    return (uint32_t)(0xFF & ~(BX - 1)) | ((uint32_t)(0xFF & ~(BY - 1)) << 8) |
           ((uint32_t)(0xFF & ~(BZ - 1)) << 16);
}
constexpr uint32_t CNT_ROUND = 65535u;
template <int BZ, bool ATOMIC>
__device__ __forceinline__ void shadow_pairs(uint32_t mine, int n, uint16_t *cnt, const DevTables &t,
                                             int R, int SR, int lane) {
    uint32_t e0 = 0, e1 = 0, cpk = 0;
    bool ylist = false;
    if (lane < n) {
        const int cx = (int)(mine & 63u) - R;
        const int cy = (int)((mine >> 6) & 31u) - R;
        const int cz = (int)((mine >> 11) & 31u) - R;
        if (cx >= -SR && cx <= BX - 1 + SR && cy >= -SR && cy <= BY - 1 + SR && cz >= -SR &&
            cz <= BZ - 1 + SR) {
            cpk = (uint32_t)(cx + 32) | ((uint32_t)(cy + 32) << 8) | ((uint32_t)(cz + 32) << 16);
            const uint32_t bin = mine >> 16;
            if (cz < 0 || cz >= BZ) {
                const uint32_t *zs = t.sh_zs + bin * (uint32_t)(2 * SR + 2);
                e0 = __ldg(zs + (max(-SR, -cz) + SR));
                e1 = __ldg(zs + (min(SR, BZ - 1 - cz) + SR + 1));
            } else if (cy < 0 || cy >= BY) {
                const uint32_t *ys = t.sh_ys + bin * (uint32_t)(2 * SR + 2);
                e0 = __ldg(ys + (max(-SR, -cy) + SR));
                e1 = __ldg(ys + (min(SR, BY - 1 - cy) + SR + 1));
                ylist = true;
            } else {
                e0 = __ldg(t.sh_start + bin);
                e1 = __ldg(t.sh_start + bin + 1);
            }
        }
    }
    for (unsigned todo = __ballot_sync(0xffffffffu, e1 > e0); todo; todo &= todo - 1u) {
        const int j = __ffs(todo) - 1;
        const uint32_t a0 = __shfl_sync(0xffffffffu, e0, j), a1 = __shfl_sync(0xffffffffu, e1, j);
        const uint32_t pk = __shfl_sync(0xffffffffu, cpk, j);
        const uint32_t *sh = __shfl_sync(0xffffffffu, (int)ylist, j) ? t.sh_y : t.sh_off;
        for (uint32_t e = a0; e < a1; e += 32) {
            const uint32_t o = e + lane < a1 ? __ldg(sh + e + lane) : SH_PAD;
            const uint32_t u = o + pk;
            if ((u & sh_inmask<BZ>()) == 0x00404040u) {
                // v = x + 32 (y + 8 z)
                const int v = (int)((u & 31u) | ((u >> 3) & 0xE0u) | ((u >> 8) & ((BZ - 1u) << 8)));
                if (ATOMIC)
                    atomicAdd(reinterpret_cast<uint32_t *>(cnt) + (v >> 1), 1u << (16 * (v & 1)));
                else
                    cnt[v] += 1;   // distinct voxels within one pair
            }
        }
        __syncwarp();              // the next pair's lanes may count the same voxels
    }
}

template <int BZ>
__device__ __forceinline__ size_t chunk_index(const DevGrid &g, int bx, int by, int bz, int row,
                                              int ch) {
    const int gy = by * BY + (row & (BY - 1)), gz = bz * BZ + row / BY;
    return ((size_t)gz * g.ny + gy) * g.pitch + (size_t)bx * BX + ch * 4;
}

__device__ __forceinline__ uint32_t codes_of(const uint4 m, uint32_t &form_bad) {
    form_bad |= (m.x & (m.x + 1u)) | (m.y & (m.y + 1u)) | (m.z & (m.z + 1u)) | (m.w & (m.w + 1u));
    return (uint32_t)__popc(m.x) | ((uint32_t)__popc(m.y) << 8) | ((uint32_t)__popc(m.z) << 16) |
           ((uint32_t)__popc(m.w) << 24);
}

__device__ __forceinline__ uint32_t apply_counts(uint2 &hv, uint2 c, uint32_t T, uint32_t Hmax) {
    const uint32_t cnt4[4] = {c.x & 0xFFFFu, c.x >> 16, c.y & 0xFFFFu, c.y >> 16};
    uint32_t h[4] = {hv.x & 0xFFFFu, hv.x >> 16, hv.y & 0xFFFFu, hv.y >> 16};
    uint32_t cross = 0;
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        const uint32_t hn = min(h[e] + cnt4[e], Hmax);
        if (cnt4[e] && h[e] < T && hn >= T) cross |= 1u << e;
        if (cnt4[e]) h[e] = hn;
    }
    hv.x = h[0] | (h[1] << 16);
    hv.y = h[2] | (h[3] << 16);
    return cross;
}

__device__ __forceinline__ void store_crossings(const DevGrid &g, size_t gi, uint32_t cross) {
    for (uint32_t m = cross; m; m &= m - 1u) g.sign[gi + (__ffs(m) - 1)] = 0u;
}

__device__ __forceinline__ void store_codes(const DevGrid &g, size_t gi, uint32_t k) {
    const uint4 m = make_uint4(code_to_mask(k & 255u), code_to_mask((k >> 8) & 255u),
                               code_to_mask((k >> 16) & 255u), code_to_mask(k >> 24));
    __stcg(reinterpret_cast<uint4 *>(g.mask + gi), m);
}

// Phase I: clears the areas [a, a + na) (no codes, zero counts), thread tid
// of gt.
template <int BZ>
__device__ __forceinline__ void clear_areas(WarpArea<BZ> *a, int na, int tid, int gt) {
    const uint4 none = make_uint4(NO_CODE4, NO_CODE4, NO_CODE4, NO_CODE4);
    const uint4 zero = make_uint4(0u, 0u, 0u, 0u);
    constexpr int K4 = brows<BZ>() * 8 / 4, C4 = bvox<BZ>() / 8;   // uint4 words of kst, cnt
    for (int v = 0; v < na; ++v) {
        uint4 *k = reinterpret_cast<uint4 *>(a[v].kst);
        uint4 *c = reinterpret_cast<uint4 *>(a[v].cnt);
        for (int i = tid; i < K4; i += gt) k[i] = none;
        for (int i = tid; i < C4; i += gt) c[i] = zero;
    }
}

// Kernel codes and shadow counts of chunk (row, ch), merged over NA areas.
template <int NA, int BZ>
__device__ __forceinline__ uint32_t chunk_codes(const WarpArea<BZ> *a, int wd) {
    uint32_t k = a[0].kst[wd];
#pragma unroll
    for (int v = 1; v < NA; ++v) k = vmin4(k, a[v].kst[wd]);
    return k;
}
template <int NA, int BZ>
__device__ __forceinline__ uint2 chunk_counts(const WarpArea<BZ> *a, int row, int ch) {
    uint2 cs = *reinterpret_cast<const uint2 *>(&a[0].cnt[row * 32 + ch * 4]);
#pragma unroll
    for (int v = 1; v < NA; ++v) {
        const uint2 cv = *reinterpret_cast<const uint2 *>(&a[v].cnt[row * 32 + ch * 4]);
        cs.x += cv.x;   // packed 16-bit counts: a voxel's total fits 16 bits
        cs.y += cv.y;
    }
    return cs;
}

// Phase D by thread tid of gt over the brick's chunks (chunk c = row * 8 +
// ch; 512 at depth 8), BATCH chunks per thread at a time: the grid masks of the chunks with
// kernel codes and the counters of the chunks with shadow counts are all
// loaded before any is used; masks are lowered to the kernel codes and
// stored where they change, counters bumped with saturation and stored, and
// the crossing voxels' signs set (Eqs. 5-6).
template <int NA, int BATCH, int BZ>
__device__ __forceinline__ void write_back(const DevGrid &g, int bx, int by, int bz,
                                           const WarpArea<BZ> *a, int tid, int gt, uint32_t T,
                                           uint32_t Hmax, uint32_t &form_bad) {
    constexpr int BCHUNKS = bchunks<BZ>();
    for (int c0 = tid; c0 < BCHUNKS; c0 += BATCH * gt) {
        uint4 m[BATCH];
        uint32_t has = 0;
#pragma unroll
        for (int q = 0; q < BATCH; ++q) {
            const int c = c0 + q * gt;
            m[q] = make_uint4(0u, 0u, 0u, 0u);
            if (c < BCHUNKS) {
                const int row = c >> 3, ch = c & 7;
                if (chunk_codes<NA>(a, kword(row, ch)) != NO_CODE4) {
                    has |= 1u << q;
                    m[q] = __ldcg(reinterpret_cast<const uint4 *>(
                        g.mask + chunk_index<BZ>(g, bx, by, bz, row, ch)));
                }
            }
        }
        uint2 hv[BATCH];
        uint32_t hc = 0;
#pragma unroll
        for (int q = 0; q < BATCH; ++q) {
            const int c = c0 + q * gt;
            hv[q] = make_uint2(0u, 0u);
            if (c < BCHUNKS) {
                const int row = c >> 3, ch = c & 7;
                const uint2 cs = chunk_counts<NA>(a, row, ch);
                if (cs.x | cs.y) {
                    hc |= 1u << q;
                    hv[q] = __ldcg(reinterpret_cast<const uint2 *>(
                        g.hits + chunk_index<BZ>(g, bx, by, bz, row, ch)));
                }
            }
        }
#pragma unroll
        for (int q = 0; q < BATCH; ++q) {
            if (!((has >> q) & 1u)) continue;
            const int c = c0 + q * gt, row = c >> 3, ch = c & 7;
            const uint32_t k = chunk_codes<NA>(a, kword(row, ch));
            const uint32_t old = codes_of(m[q], form_bad);
            const uint32_t lt = code_lt(old, k);
            if (lt) store_codes(g, chunk_index<BZ>(g, bx, by, bz, row, ch), code_min(old, k, lt));
        }
#pragma unroll
        for (int q = 0; q < BATCH; ++q) {
            if (!((hc >> q) & 1u)) continue;
            const int c = c0 + q * gt, row = c >> 3, ch = c & 7;
            const size_t gi = chunk_index<BZ>(g, bx, by, bz, row, ch);
            const uint32_t cross = apply_counts(hv[q], chunk_counts<NA>(a, row, ch), T, Hmax);
            __stcg(reinterpret_cast<uint2 *>(g.hits + gi), hv[q]);
            store_crossings(g, gi, cross);
        }
    }
}

// Phase D of a light brick, by one warp.  Lane l visits chunk i (i < NI) at
// row 4 i + l / 8, word (l + i) mod 8: every chunk once, and a kernel box's
// few covered words of a row fall to different lanes in different rows, so
// each lane holds about the same number of covered chunks (with lanes fixed
// to a word, the lanes of the covered words would walk every row while the
// others idle).  The covered chunks (those with kernel codes; a chunk with
// shadow counts lies in its contact's K^3 box and so has codes too) are
// noted in a bit mask first, then taken WBL_PICKS per lane at a time: their
// masks and counters loaded together, then lowered, bumped and stored as in
// write_back (three at a time measured fastest: more keep more registers
// live across the loads).
constexpr int WBL_PICKS = 3;
template <int BZ>
__device__ __forceinline__ void write_back_light(const DevGrid &g, int bx, int by, int bz,
                                                 const WarpArea<BZ> *a, int lane, uint32_t T,
                                                 uint32_t Hmax, uint32_t &form_bad) {
    constexpr int NI = bchunks<BZ>() / 32;
    static_assert(NI <= 32, "one bit per visited chunk");
    uint32_t cov = 0;
#pragma unroll
    for (int i = 0; i < NI; ++i) {
        const int row = 4 * i + (lane >> 3), ch = (lane + i) & 7;
        if (a->kst[kword(row, ch)] != NO_CODE4) cov |= 1u << i;
    }
    while (__any_sync(0xffffffffu, cov != 0u)) {
        int rc[WBL_PICKS];                            // row * 8 + ch of each taken chunk, -1 = none
        uint4 m[WBL_PICKS];
#pragma unroll
        for (int q = 0; q < WBL_PICKS; ++q) {
            rc[q] = -1;
            m[q] = make_uint4(0u, 0u, 0u, 0u);
            if (cov) {
                const int i = __ffs(cov) - 1;
                cov &= cov - 1u;
                const int row = 4 * i + (lane >> 3), ch = (lane + i) & 7;
                rc[q] = row * 8 + ch;
                m[q] = __ldcg(reinterpret_cast<const uint4 *>(g.mask + chunk_index<BZ>(g, bx, by, bz, row, ch)));
            }
        }
        uint2 hv[WBL_PICKS];
        uint32_t hc = 0;
#pragma unroll
        for (int q = 0; q < WBL_PICKS; ++q) {
            hv[q] = make_uint2(0u, 0u);
            if (rc[q] >= 0) {
                const uint2 cs = chunk_counts<1>(a, rc[q] >> 3, rc[q] & 7);
                if (cs.x | cs.y) {
                    hc |= 1u << q;
                    hv[q] = __ldcg(reinterpret_cast<const uint2 *>(
                        g.hits + chunk_index<BZ>(g, bx, by, bz, rc[q] >> 3, rc[q] & 7)));
                }
            }
        }
#pragma unroll
        for (int q = 0; q < WBL_PICKS; ++q) {
            if (rc[q] < 0) continue;
            const int row = rc[q] >> 3, ch = rc[q] & 7;
            const uint32_t k = a->kst[kword(row, ch)];
            const uint32_t old = codes_of(m[q], form_bad);
            const uint32_t lt = code_lt(old, k);
            if (lt) store_codes(g, chunk_index<BZ>(g, bx, by, bz, row, ch), code_min(old, k, lt));
        }
#pragma unroll
        for (int q = 0; q < WBL_PICKS; ++q) {
            if (!((hc >> q) & 1u)) continue;
            const int row = rc[q] >> 3, ch = rc[q] & 7;
            const size_t gi = chunk_index<BZ>(g, bx, by, bz, row, ch);
            const uint32_t cross = apply_counts(hv[q], chunk_counts<1>(a, row, ch), T, Hmax);
            __stcg(reinterpret_cast<uint2 *>(g.hits + gi), hv[q]);
            store_crossings(g, gi, cross);
        }
    }
}

// ---------------------------------------------------------------- dense bricks
// For a brick with many pairs, the Eq. 4 result is computed once per voxel
// instead of once per pair: the mask left by AND-ing the kernels of all
// contacts c whose K^3 window holds voxel v is the mask of code
// ceil(sqrt(f(v))) with f(v) = min |v - c|^2 over those contacts, and this
// windowed minimum separates along the axes:
//   f = min_{|dz|<=R} [dz^2 + min_{|dy|<=R} [dy^2 + min_{|dx|<=R} dx^2]]
// where the innermost minimum runs over the contacts of one row.  Rows of the
// brick dilated by R hold 64-bit contact occupancy masks; pass x finds the
// nearest contact within +-R of each voxel by bit scans, passes y and z are
// 2R+1-tap min-plus sweeps on bytes, four voxels per word.  With R <= 6 every
// finite sum is at most 3 R^2 = 108, and the no-contact value DENSE_INF = 127
// plus a tap stays below 256, so bytes never carry into each other.
constexpr uint32_t DENSE_INF = 127u;
// The dense path's scratch (occupancy, two passes, plane masks, row list)
// lives in the warp areas of the heavy group after the first: at R = 6 all
// eight warps form the group; up to R = 5 four do (three spare areas).
__host__ __device__ constexpr int dense_scratch_bytes(int R, int BZ) {
    return 8 * (BY + 2 * R) * (BZ + 2 * R) + 32 * (BY + 2 * R) * (BZ + 2 * R) +
           4 * 8 * BY * (BZ + 2 * R) + 4 * (BZ + 2 * R) + 4 + 2 * (BY + 2 * R) * (BZ + 2 * R);
}
// Largest R whose dense scratch fits a half group's three spare areas (the
// half-group split is used up to R = 5 where it fits).
template <int BZ> __host__ __device__ constexpr int half_group_max_r() { return BZ == 4 ? 3 : 5; }
template <int BZ>
__host__ __device__ constexpr bool dense_scratch_fits() {
    return dense_scratch_bytes(6, BZ) <= (WPC - 1) * (int)sizeof(WarpArea<BZ>) &&
           dense_scratch_bytes(half_group_max_r<BZ>(), BZ) <= (WPC / 2 - 1) * (int)sizeof(WarpArea<BZ>);
}
static_assert(dense_scratch_fits<4>() && dense_scratch_fits<8>() && dense_scratch_fits<16>(),
              "dense scratch: R = 6 in seven spare areas, half groups in three");
static_assert(BZ_MAX + 2 * 6 <= 32, "dense path: one bit per dilated plane in a 32-bit mask");

// Run by a heavy group of gt threads (gw = gt / 32 warps); tid is the
// thread's index in the group, areas the group's first warp area, and the
// group synchronises on named barrier bar.  The codes of area 0 are all
// written by pass z (32 where no contact's window reaches), its counts
// cleared here.
template <int BZ>
__device__ void integrate_dense(const DevGrid &g, int bx, int by, int bz, const uint32_t *pairs,
                                uint32_t len, WarpArea<BZ> *areas, const uint8_t *ctab,
                                const DevTables &t, int R, int SR,
                                uint32_t T, uint32_t Hmax, uint32_t &form_bad, int tid, int gt,
                                int bar) {
    const int lane = tid & 31, warp = tid >> 5, gw = gt >> 5;
    const int DY = BY + 2 * R, DZ = BZ + 2 * R;                 // dilated y / z extents
    unsigned char *scr = reinterpret_cast<unsigned char *>(areas + 1);
    unsigned long long *occ = reinterpret_cast<unsigned long long *>(scr);   // DZ x DY rows
    uint32_t *g1 = reinterpret_cast<uint32_t *>(scr + DY * DZ * 8);        // DZ x DY rows x 8 words
    uint32_t *g2 = g1 + DY * DZ * 8;                                        // DZ x BY rows x 8 words
    uint32_t *pmask = g2 + DZ * BY * 8;    // per dilated plane z: bit y = row (y, z) has a contact
    uint32_t *nlist = pmask + DZ;          // number of rows with a contact
    uint16_t *list = reinterpret_cast<uint16_t *>(nlist + 1);              // those rows
    WarpArea<BZ> *a0 = areas;
    const uint32_t inf4 = DENSE_INF * 0x01010101u;
    // clear the counts and the occupancy
    {
        uint4 *c = reinterpret_cast<uint4 *>(a0->cnt);
        for (int i = tid; i < bvox<BZ>() / 8; i += gt) c[i] = make_uint4(0u, 0u, 0u, 0u);
    }
    for (int r = tid; r < DY * DZ; r += gt) occ[r] = 0ull;
    if (tid < DZ) pmask[tid] = 0u;
    if (tid == 0) *nlist = 0u;
    group_sync(bar, gt);
    // contacts: payload coordinates are brick-relative + R, i.e. dilated indices
    for (uint32_t j = tid; j < len; j += gt) {
        const uint32_t pl = __ldg(pairs + j);
        atomicOr(&occ[((pl >> 11) & 31u) * DY + ((pl >> 6) & 31u)], 1ull << (pl & 63u));
    }
    group_sync(bar, gt);
    // rows without a contact are all INF after pass x: write them directly,
    // list the others, and note per plane which rows hold contacts
    for (int r = tid; r < DY * DZ; r += gt) {
        if (occ[r]) {
            atomicOr(&pmask[r / DY], 1u << (r % DY));
            list[atomicAdd(nlist, 1u)] = (uint16_t)r;
        } else {
            uint4 *row = reinterpret_cast<uint4 *>(g1 + r * 8);
            row[0] = make_uint4(inf4, inf4, inf4, inf4);
            row[1] = make_uint4(inf4, inf4, inf4, inf4);
        }
    }
    group_sync(bar, gt);
    // pass x over the listed rows: squared distance to the nearest contact of
    // the row within +-R
    const uint32_t win = (1u << (2 * R + 1)) - 1u, lmask = (1u << (R + 1)) - 1u;
    const uint32_t nl = *nlist;
    for (uint32_t i = warp; i < nl; i += gw) {
        const int r = list[i];
        const unsigned long long o = occ[r];
        uint32_t v = DENSE_INF;
        const uint32_t wv = (uint32_t)(o >> lane) & win;   // bit j: contact at x - R + j
        const uint32_t left = wv & lmask, right = wv >> R;
        int d = 2 * R + 2;
        if (left) d = R - (31 - __clz(left));
        if (right) d = min(d, __ffs(right) - 1);
        if (d <= R) v = (uint32_t)(d * d);
        reinterpret_cast<unsigned char *>(g1)[r * 32 + lane] = (unsigned char)v;
    }
    group_sync(bar, gt);
    // pass y: taps only from rows with contacts (an INF row cannot lower the
    // minimum: INF + dy^2 >= INF and the result is clamped to INF)
    const uint32_t twin = (1u << (2 * R + 1)) - 1u;
    static_assert(BY == 8, "pass y indexes brick rows y by 3 bits");
    for (int idx = tid; idx < DZ * BY * 8; idx += gt) {
        const int w = idx & 7, y = (idx >> 3) & 7, zp = idx >> 6;
        uint32_t acc = inf4;
        for (uint32_t m = (pmask[zp] >> y) & twin; m; m &= m - 1u) {
            const int t = __ffs(m) - 1, dy = t - R;
            acc = vmin4(acc, g1[(zp * DY + (y + t)) * 8 + w] + (uint32_t)(dy * dy) * 0x01010101u);
        }
        g2[(zp * 8 + y) * 8 + w] = vmin4(acc, inf4);
    }
    uint32_t planes = 0;                   // planes with any contact
    for (int zp = 0; zp < DZ; ++zp) planes |= (pmask[zp] ? 1u : 0u) << zp;
    group_sync(bar, gt);
    // pass z (taps only from planes with contacts) and the codes: the
    // minimum kernel code of every voxel of the brick
    for (int idx = tid; idx < brows<BZ>() * 8; idx += gt) {
        const int w = idx & 7, row = idx >> 3, y = row & 7, z = row >> 3;
        uint32_t acc = inf4;
        for (uint32_t m = (planes >> z) & twin; m; m &= m - 1u) {
            const int t = __ffs(m) - 1, dz = t - R;
            acc = vmin4(acc, g2[((z + t) * 8 + y) * 8 + w] + (uint32_t)(dz * dz) * 0x01010101u);
        }
        a0->kst[kword(row, w)] = (uint32_t)ctab[acc & 255u] | ((uint32_t)ctab[(acc >> 8) & 255u] << 8) |
                                 ((uint32_t)ctab[(acc >> 16) & 255u] << 16) |
                                 ((uint32_t)ctab[acc >> 24] << 24);
    }
    // Eq. 5 counts into one array: warp w takes an equal share of the pairs
    // (len * w / gw onwards), 32 at a time; the phase ends at the barrier
    // below, so the largest share sets its length
    const uint32_t jlo = len * (uint32_t)warp / (uint32_t)gw;
    const uint32_t jhi = len * (uint32_t)(warp + 1) / (uint32_t)gw;
    for (uint32_t j0 = jlo; j0 < jhi; j0 += 32u) {
        const uint32_t mine = j0 + lane < jhi ? __ldg(pairs + j0 + lane) : 0u;
        shadow_pairs<BZ, true>(mine, (int)min(32u, jhi - j0), a0->cnt, t, R, SR, lane);
    }
    group_sync(bar, gt);
    write_back<1, 2>(g, bx, by, bz, a0, tid, gt, T, Hmax, form_bad);
}

// Grid of global brick b in a batch (bricks of grid m are [bbase[m], bbase[m+1])).
__device__ __forceinline__ int grid_of_brick(const BatchDev &bd, uint32_t b) {
    int lo = 0, hi = bd.n_grids - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (bd.bbase[mid] <= b) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// Grid view and local brick index of touched brick b.
template <bool BATCH>
__device__ __forceinline__ uint32_t brick_grid(const DevGrid &g, const BatchDev &bd, uint32_t b,
                                               DevGrid &gg) {
    if (!BATCH) {
        gg = g;
        return b;
    }
    const int gi = grid_of_brick(bd, b);
    gg = bd.grids[gi];
    return b - bd.bbase[gi];
}

template <int NW, bool BATCH, int BZ>
__global__ void __launch_bounds__(NTHR, 4) k_integrate(DevGrid g0, BatchDev bd, DevParams p,
                                                    DevTables t, long long n_input, WsDev ws) {
    extern __shared__ __align__(16) uint32_t smem[];
    __shared__ uint32_t s_item[2];                        // per heavy group
    __shared__ uint32_t s_vitem;                          // the CTA's very heavy brick
    __shared__ uint8_t s_ctab[256];
    for (int j = threadIdx.x; j < 256; j += NTHR) {
        int kk = 0;
        while (kk * kk < j && kk < 16) ++kk;
        s_ctab[j] = (uint8_t)(j < (int)DENSE_INF ? kk : 32);   // ceil(sqrt(f)); 32 = no change
    }
    const int R = p.R;
    const int W = 2 * R + 4;
    const int np = (2 * R * R + 1) * W;
    uint32_t *P = smem;
    for (int j = threadIdx.x; j < np; j += NTHR) P[j] = t.prow[j];
    WarpArea<BZ> *areas = reinterpret_cast<WarpArea<BZ> *>(smem + ((np + 3) & ~3));
    // shadow offset lists stay in global memory (read-only path,
    // L1-resident): the shared memory they would take costs a CTA per SM
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    WarpArea<BZ> *wa = areas + warp;
    // the tables above are the kernels' own; the workspace is the previous
    // kernels' output
    pdl_wait();
    pdl_launch_dependents();
    const uint32_t nt = min(*(volatile uint32_t *)&ws.hdr->n_touched, ws.max_touched);
    const uint32_t nvheavy = *(volatile uint32_t *)&ws.hdr->n_vheavy;
    const uint32_t nheavy = min(*(volatile uint32_t *)&ws.hdr->n_heavy + nvheavy, nt);

    const int SR = p.sr;
    const uint32_t T = (uint32_t)p.T, Hmax = (uint32_t)p.Hmax;
    uint32_t form_bad = 0;

    // ---------------- work: heavy bricks by groups of hw warps, light ones by single warps
    // At K <= 11 (K <= 7 for BZ = 4) the dense path runs on groups of four
    // warps (its scratch fits a group's three spare areas): the very heavy
    // bricks are taken first by whole CTAs (their Eq. 5 counts grow with the
    // pairs, so on four warps the largest would outlast the launch), then
    // group 0 (warps 0-3) takes heavy bricks first, group 1 (warps 4-7) light
    // bricks first, so the largest light bricks start at the beginning of the
    // launch instead of after the heavy ones; each group then turns to the
    // other kind.  Otherwise the whole CTA is one group, heavy bricks (very
    // heavy first) first.
    const int hw = (NW == 4 && R <= half_group_max_r<BZ>()) ? WPC / 2 : WPC;
    const int ht = hw * 32;
    const int gidx = warp / hw;                  // group of this warp
    const int gtid = tid - gidx * ht, gwarp = warp - gidx * hw;
    const int gbar = 1 + gidx;                   // its named barrier
    WarpArea<BZ> *garea = areas + gidx * hw;     // its first warp area
    // First claims are static (heavy item f for group 0, light item f * hw +
    // gwarp for group 1's warps, f = the CTA's rank among those that do not
    // start on a very heavy brick): a launch's thousands of warps claiming at
    // once through one counter would wait on each other's atomics.  The CTAs
    // that start on a very heavy brick (the first nv_cta) claim through the
    // counters only, so the largest light bricks are not held back until
    // they finish.  Later claims take counter values past the static ranges.
    const uint32_t nv_cta = hw < WPC ? min(nvheavy, gridDim.x) : 0u;
    const uint32_t n_free = gridDim.x - nv_cta, f = blockIdx.x - nv_cta;
    const uint32_t n_static_heavy = n_free;
    const uint32_t n_static_light = hw < WPC ? n_free * (uint32_t)(WPC - hw) : 0u;
    bool first_heavy = gidx == 0 && blockIdx.x >= nv_cta, first_light = gidx == 1 && blockIdx.x >= nv_cta;
    // heavy items [h0, nheavy) go to the groups; items < nvheavy are the very
    // heavy bricks (back of order)
    const uint32_t h0 = hw < WPC ? nvheavy : 0u;
    __syncthreads();                             // tables above, for every warp
    if constexpr (NW == 4) {
        // very heavy bricks by whole CTAs: item blockIdx.x first, then counter
        // values past the grid
        for (uint32_t it = hw < WPC ? blockIdx.x : nvheavy; it < nvheavy;) {
            const uint32_t b = ws.order[ws.max_touched - 1 - it];
            const uint32_t start = ws.boff[b];
            uint32_t len = ws.bcnt[b];
            if ((unsigned long long)start + len > ws.pairs_cap) len = 0;   // cannot happen by sizing
            DevGrid g;
            const uint32_t lb = brick_grid<BATCH>(g0, bd, b, g);
            const int bx = (int)(lb % (uint32_t)g.nbx);
            const uint32_t byz = lb / (uint32_t)g.nbx;
            const int by = (int)(byz % (uint32_t)g.nby), bz = (int)(byz / (uint32_t)g.nby);
            for (uint32_t r0 = 0; r0 < len; r0 += CNT_ROUND) {
                integrate_dense(g, bx, by, bz, ws.pairs + start + r0, min(len - r0, CNT_ROUND), areas,
                                s_ctab, t, R, SR, T, Hmax, form_bad, tid, NTHR, 0);
                __syncthreads();
            }
            if (tid == 0) {
                ws.bcnt[b] = 0u;
                s_vitem = gridDim.x + atomicAdd(&ws.hdr->next_vheavy, 1u);
            }
            __syncthreads();
            it = s_vitem;   // written again only after the next brick's barriers
        }
    }
    for (int phase = 0; phase < 2; ++phase) {
        if ((phase == 0) == (gidx == 0)) {
            // heavy bricks, one per group
            for (;;) {
                group_sync(gbar, ht);
                if (gtid == 0)
                    s_item[gidx] = h0 + (first_heavy ? f
                                                     : n_static_heavy + atomicAdd(&ws.hdr->next_heavy, 1u));
                first_heavy = false;
                group_sync(gbar, ht);
                const uint32_t it = s_item[gidx];
                if (it >= nheavy) break;
                // the very heavy bricks (back of order) first
                const uint32_t b = it < nvheavy ? ws.order[ws.max_touched - 1 - it] : ws.order[it - nvheavy];
                const uint32_t start = ws.boff[b];
                uint32_t len = ws.bcnt[b];
                if ((unsigned long long)start + len > ws.pairs_cap) len = 0;   // cannot happen by sizing
                DevGrid g;
                const uint32_t lb = brick_grid<BATCH>(g0, bd, b, g);
                const int bx = (int)(lb % (uint32_t)g.nbx);
                const uint32_t byz = lb / (uint32_t)g.nbx;
                const int by = (int)(byz % (uint32_t)g.nby), bz = (int)(byz / (uint32_t)g.nby);
                const uint32_t *pairs = ws.pairs + start;

                // the pairs in rounds of at most CNT_ROUND, so that no count can
                // pass 2^16 (group-uniform: every thread sees the same len)
                for (uint32_t r0 = 0; r0 < len; r0 += CNT_ROUND) {
                    const uint32_t *rp = pairs + r0;
                    const uint32_t rl = min(len - r0, CNT_ROUND);
                    if constexpr (NW == 4) {
                        integrate_dense(g, bx, by, bz, rp, rl, garea, s_ctab, t, R, SR, T, Hmax,
                                        form_bad, gtid, ht, gbar);
                        group_sync(gbar, ht);
                        continue;
                    }
                    // I: every warp's area
                    clear_areas(garea, hw, gtid, ht);
                    group_sync(gbar, ht);
                    // C: warp w applies pairs w, w + WPC, w + 2 WPC, ... to its own area
                    for (uint32_t base = 0; base * WPC + warp < rl; base += 32) {
                        const uint32_t jj = (base + lane) * WPC + warp;
                        const uint32_t mine = jj < rl ? __ldg(rp + jj) : 0u;
                        const int cnt = (int)min(32u, (rl - warp + WPC - 1) / WPC - base);
                        const RowsSetup su = rows_setup<BZ>(mine, R);    // lanes >= cnt: unused
                        for (int j = 0; j < cnt; ++j) {
                            const RowsSetup sj = {__shfl_sync(0xffffffffu, su.a, j),
                                                  __shfl_sync(0xffffffffu, su.b, j)};
                            apply_rows<NW, BZ>(sj, wa, P, W, lane);
                            __syncwarp();
                        }
                        shadow_pairs<BZ, false>(mine, cnt, wa->cnt, t, R, SR, lane);
                    }
                    group_sync(gbar, ht);
                    // D: the areas merged (byte-wise min of codes, sum of counts) and written back
                    write_back<WPC, 2>(g, bx, by, bz, garea, gtid, ht, T, Hmax, form_bad);
                    group_sync(gbar, ht);
                }
                if (gtid == 0) ws.bcnt[b] = 0u;
            }
        } else {
            // light bricks, one per warp
            for (;;) {
                uint32_t w = 0;
                if (first_light) {
                    w = f * (uint32_t)hw + (uint32_t)gwarp;
                    first_light = false;
                } else {
                    if (lane == 0) w = atomicAdd(&ws.hdr->next_work, 1u);
                    w = n_static_light + __shfl_sync(0xffffffffu, w, 0);
                }
                if (nheavy + w >= nt) break;
                // the larger size classes first (the class sizes are fixed during
                // the launch: plain loads, served from L1 after the first)
                int c = 0;
                uint32_t q = w;
#pragma unroll
                for (int k = 0; k < LIGHT_CLASSES - 1; ++k) {
                    const uint32_t nk = ws.hdr->n_cls[k];
                    if (c == k && q >= nk) {
                        q -= nk;
                        c = k + 1;
                    }
                }
                const uint32_t b = *light_queue_slot(ws, c, q);
                const uint32_t start = ws.boff[b];
                uint32_t len = ws.bcnt[b];
                if ((unsigned long long)start + len > ws.pairs_cap) len = 0;   // cannot happen by sizing
                DevGrid g;
                const uint32_t lb = brick_grid<BATCH>(g0, bd, b, g);
                const int bx = (int)(lb % (uint32_t)g.nbx);
                const uint32_t byz = lb / (uint32_t)g.nbx;
                const int by = (int)(byz % (uint32_t)g.nby), bz = (int)(byz / (uint32_t)g.nby);
                const uint32_t *pairs = ws.pairs + start;

                for (uint32_t r0 = 0; r0 < len; r0 += CNT_ROUND) {   // rounds as for heavy bricks
                    const uint32_t *rp = pairs + r0;
                    const uint32_t rl = min(len - r0, CNT_ROUND);
                    // I
                    clear_areas(wa, 1, lane, 32);
                    __syncwarp();
                    // C
                    for (uint32_t base = 0; base < rl; base += 32) {
                        const uint32_t mine = base + lane < rl ? __ldg(rp + base + lane) : 0u;
                        const int cnt = (int)min(32u, rl - base);
                        const RowsSetup su = rows_setup<BZ>(mine, R);    // lanes >= cnt: unused
                        for (int j = 0; j < cnt; ++j) {
                            const RowsSetup sj = {__shfl_sync(0xffffffffu, su.a, j),
                                                  __shfl_sync(0xffffffffu, su.b, j)};
                            apply_rows<NW, BZ>(sj, wa, P, W, lane);
                            __syncwarp();
                        }
                        shadow_pairs<BZ, false>(mine, cnt, wa->cnt, t, R, SR, lane);
                    }
                    // D
                    __syncwarp();
                    write_back_light<BZ>(g, bx, by, bz, wa, lane, T, Hmax, form_bad);
                    __syncwarp();
                }
                if (lane == 0) ws.bcnt[b] = 0u;
                __syncwarp();
            }
        }
    }
    if (form_bad) atomicOr(&ws.hdr->err, ERR_MASK_FORM);

    // Last warp out publishes the scan's counters and re-arms the workspace.
    if (lane == 0) {
        __threadfence();
        if (atomicAdd(&ws.hdr->done_ctas, 1u) == gridDim.x * WPC - 1) {
            __threadfence();
            WsHeader *h = ws.hdr;
            volatile WsHeader *vh = h;
            h->last.n_input = n_input;
            h->last.n_valid = (long long)vh->acc_valid;
            h->last.n_inside = (long long)vh->acc_inside;
            h->last.n_kept = (long long)vh->acc_kept;
            h->last.n_pairs = (long long)vh->pool;
            h->last.n_bricks = (long long)vh->n_touched;
            h->last.error = atomicOr(&h->err, 0u);
            h->last.reserved = 0u;
            if (ws.stats_out) *ws.stats_out = h->last;      // written through to host memory
            h->err = 0u;
            h->n_touched = 0u;
            h->pool = 0u;
            h->next_work = 0u;
            h->n_heavy = 0u;
            h->n_vheavy = 0u;
            for (int c = 0; c < LIGHT_CLASSES; ++c) h->n_cls[c] = 0u;
            h->next_heavy = 0u;
            h->next_vheavy = 0u;
            h->acc_valid = 0ull;
            h->acc_inside = 0ull;
            h->acc_kept = 0ull;
            __threadfence();
            h->done_ctas = 0u;
        }
    }
}

// Dynamic shared memory of one CTA: row codes and warp areas.
static size_t integrate_smem(int K, int bz) {
    const int R = (K - 1) / 2;
    const size_t np = (size_t)(2 * R * R + 1) * (2 * R + 4);
    const size_t area = bz == 4 ? sizeof(WarpArea<4>) : bz == 16 ? sizeof(WarpArea<16>)
                                                                  : sizeof(WarpArea<8>);
    return ((np + 3) & ~size_t(3)) * 4 + WPC * area;
}

// Launch configuration, cached per device.  Calls for different devices or
// workspaces may come from several host threads, so the cache is guarded.
constexpr int kCfgDevices = 64;
struct IntegrateCfg {
    bool limits_set[3][2] = {};         // per depth: shared-memory limit raised (4-word, 6-word rows)
    int ctas[3][MAX_K + 1] = {};
};
static IntegrateCfg g_cfg[kCfgDevices];
static std::mutex g_cfg_mutex;

// Occupancy-based persistent grid for one kernel size; the shared-memory
// limit of each template instance is raised once per device to what its
// largest kernel size needs (the attribute belongs to the function, so it
// must not be lowered for a smaller K).
template <int NW, int BZ>
static int configure(int dev, bool &limits_set, size_t smem, size_t smem_max) {
    int sms = 0, per_sm = 0;
    if (!limits_set) {
        cudaFuncSetAttribute(k_integrate<NW, false, BZ>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem_max);
        cudaFuncSetAttribute(k_integrate<NW, true, BZ>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem_max);
        limits_set = true;
    }
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_integrate<NW, true, BZ>, NTHR, smem);
    return max(1, sms * max(1, per_sm));
}

// Words of a kernel row: an x-extent of K voxels starting anywhere in a word.
static int words_per_row(int K) { return K <= 13 ? 4 : 6; }

int device_sm_count() {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms > 0 ? sms : 1;
}

template <int BZ>
static int configure_depth(int dev, bool limits_set[2], int K) {
    const size_t smem = integrate_smem(K, BZ);
    if (words_per_row(K) == 4) return configure<4, BZ>(dev, limits_set[0], smem, integrate_smem(13, BZ));
    const int kmax = BZ == 16 ? BZ16_MAX_K : MAX_K;
    return configure<6, BZ>(dev, limits_set[1], smem, integrate_smem(kmax, BZ));
}

// Persistent grid for these parameters and brick depth: every SM filled to
// its occupancy limit.
int integrate_grid_ctas(const DevParams &p, int bz) {
    int dev = 0;
    cudaGetDevice(&dev);
    IntegrateCfg local;                                 // devices past the cache: not cached
    IntegrateCfg &c = (dev >= 0 && dev < kCfgDevices) ? g_cfg[dev] : local;
    const int d = bz_shift(bz) - 2;
    std::lock_guard<std::mutex> lock(g_cfg_mutex);
    if (!c.ctas[d][p.K]) {
        c.ctas[d][p.K] = d == 0   ? configure_depth<4>(dev, c.limits_set[0], p.K)
                         : d == 2 ? configure_depth<16>(dev, c.limits_set[2], p.K)
                                  : configure_depth<8>(dev, c.limits_set[1], p.K);
    }
    return c.ctas[d][p.K];
}

template <bool BATCH, int BZ>
static void launch_depth(const DevGrid &g, const BatchDev &bd, const DevParams &p, const DevTables &t,
                         long long n_input, const WsDev &ws, int grid_ctas, cudaStream_t s) {
    const size_t smem = integrate_smem(p.K, BZ);
    if (words_per_row(p.K) == 4)
        launch_pdl(k_integrate<4, BATCH, BZ>, grid_ctas, NTHR, smem, s, g, bd, p, t, n_input, ws);
    else
        launch_pdl(k_integrate<6, BATCH, BZ>, grid_ctas, NTHR, smem, s, g, bd, p, t, n_input, ws);
}

template <bool BATCH>
static void launch_any(int bzs, const DevGrid &g, const BatchDev &bd, const DevParams &p,
                       const DevTables &t, long long n_input, const WsDev &ws, int grid_ctas,
                       cudaStream_t s) {
    if (bzs == 2) launch_depth<BATCH, 4>(g, bd, p, t, n_input, ws, grid_ctas, s);
    else if (bzs == 4) launch_depth<BATCH, 16>(g, bd, p, t, n_input, ws, grid_ctas, s);
    else launch_depth<BATCH, 8>(g, bd, p, t, n_input, ws, grid_ctas, s);
}

void launch_integrate(const DevGrid &g, const DevParams &p, const DevTables &t, long long n_input,
                      const WsDev &ws, int grid_ctas, cudaStream_t s) {
    launch_any<false>(g.bzs, g, BatchDev{}, p, t, n_input, ws, grid_ctas, s);
}

void launch_integrate_batch(const BatchDev &bd, const DevParams &p, const DevTables &t,
                            long long n_input, const WsDev &ws, int grid_ctas, cudaStream_t s) {
    launch_any<true>(bd.bzs, DevGrid{}, bd, p, t, n_input, ws, grid_ctas, s);
}

// ---------------------------------------------------------------- op-rate micro-benchmark
// Peak rates of the two shared-memory updates the brick integration is built
// from, each measured alone at the integration's occupancy (4 CTAs of 256
// threads per SM): the op-side ceiling of the roofline (Eq. 7: the update
// time is the number of elementary updates times their cost).
//   MODE 0, 1: Eq. 4 on packed codes: a kernel-row table word and a staged
//              4-voxel word loaded from shared memory and their byte-wise
//              minimum (code_lt / code_min) stored back, always (0) or only
//              when it changes the word (1; the table words are then never
//              below the staged ones); 4 voxel-ANDs per update.
//   MODE 2:    Eq. 5 counts: a staged 16-bit counter incremented.
// Every lane works in words of its own bank (no conflicts); the unrolled
// inner loop leaves issue, not loop overhead, as the limit.  The staged
// words are accessed through a volatile pointer, so that every update
// loads and stores shared memory as the integration's do (a thread's own
// word would otherwise stay in a register across the loop).
constexpr int OP_WORDS = 4;
template <int MODE>
__global__ void __launch_bounds__(NTHR, 4) k_op_rate(int iters, unsigned long long *sink) {
    __shared__ uint32_t s_tab_[8 * NTHR];
    __shared__ uint32_t s_st_[OP_WORDS * NTHR];
    volatile uint32_t *s_tab = s_tab_;
    volatile uint32_t *s_st = s_st_;
    const int tid = threadIdx.x;
    for (int j = 0; j < 8; ++j)
        s_tab[j * NTHR + tid] = MODE == 1 ? 0x20202020u : 0x01010101u * (uint32_t)((tid + j) % 30 + 1);
    for (int w = 0; w < OP_WORDS; ++w) s_st[w * NTHR + tid] = MODE == 1 ? 0x10101010u : 0x1F1F1F1Fu;
    __syncthreads();
    uint32_t acc = 0;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int w = 0; w < OP_WORDS; ++w) {
            const int ti = ((it * OP_WORDS + w) & 7) * NTHR + tid, si = w * NTHR + tid;
            if constexpr (MODE == 2) {
                volatile uint16_t *c = reinterpret_cast<volatile uint16_t *>(s_st) + 2 * si;
                *c = (uint16_t)(*c + 1u);
            } else {
                const uint32_t kwd = s_tab[ti];
                const uint32_t a = s_st[si];
                const uint32_t lt = code_lt(a, kwd);
                if (MODE == 0 || lt) s_st[si] = code_min(a, kwd, lt);
                acc += lt;
            }
        }
    }
    __syncthreads();
    for (int w = 0; w < OP_WORDS; ++w) acc += s_st[w * NTHR + tid];
    if (acc == 0x9E3779B9u) atomicAdd(sink, 1ull);     // keeps the loop; practically never true
}

}  // namespace dbt

using namespace dbt;

extern "C" dbt_status dbt_op_rates(int32_t iters, double *and_per_s, double *count_per_s) {
    if (iters < 16 || iters > (1 << 24) || !and_per_s || !count_per_s) {
        return report_einval("dbt_op_rates: iters in [16, 2^24] and non-NULL outputs");
    }
    const int ctas = device_sm_count() * 4;
    unsigned long long *sink = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaMalloc(&sink, sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    float ms[3] = {0.f, 0.f, 0.f};
    for (int mode = 0; mode < 3 && e == cudaSuccess; ++mode) {
        for (int rep = 0; rep < 2 && e == cudaSuccess; ++rep) {     // the first run warms up
            cudaEventRecord(e0, 0);
            if (mode == 0) k_op_rate<0><<<ctas, NTHR>>>(iters, sink);
            else if (mode == 1) k_op_rate<1><<<ctas, NTHR>>>(iters, sink);
            else k_op_rate<2><<<ctas, NTHR>>>(iters, sink);
            cudaEventRecord(e1, 0);
            e = cudaEventSynchronize(e1);
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms[mode], e0, e1);
        }
    }
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (sink) cudaFree(sink);
    if (e != cudaSuccess) return report_cuda_error(e, "dbt_op_rates");
    const double updates = (double)ctas * NTHR * (double)iters * OP_WORDS;
    const double best_and_ms = std::min(ms[0], ms[1]);
    *and_per_s = 4.0 * updates / (best_and_ms * 1e-3);
    *count_per_s = updates / (ms[2] * 1e-3);
    return DBT_OK;
}
