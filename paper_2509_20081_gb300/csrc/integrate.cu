// Brick integration of one scan (Sec. III-C, Eqs. 4-6).
//
// Persistent CTAs of WPC warps; each warp takes touched bricks (32 x 8 x 8
// voxels) from a dynamic queue and owns its brick alone, so no two threads
// of different warps ever touch the same voxel and no atomics are needed.
//
// Distance codes.  A mask of the form 2^k - 1 is stored as k = popcount; the
// Eq. 4 AND of two such masks is the mask of min(k).  Grid masks start all
// ones (Sec. III-A) and only ever meet Eq. 3 masks, so they keep this form
// (checked on load; a violation latches ERR_MASK_FORM).  Staged bricks hold
// 8-bit codes, four voxels per 32-bit word, and the AND of four voxels is
// one byte-wise minimum.
//
// Kernel rows.  For a row of the K^3 kernel at squared lateral offset
// q = oy^2 + oz^2, the codes along x are ceil(sqrt(ox^2 + q)).  The host
// builds P[q][s]: the four codes a 4-voxel word receives when its first
// voxel sits at ox = s - 3 - R (32 = no change outside the kernel).  One
// word update is then a table load, a load of the staged word, a byte-wise
// min and a conditional store.
//
// Per brick the warp
//   A. ORs, per brick row, the 16-byte chunks any return's kernel covers,
//   B. stages those chunks as codes (and zeroes per-voxel shadow counts),
//   C. applies every (return, brick) pair: one warp iteration per kernel
//      plane (lanes = 8 rows x 4 words), then the bin's shadow offsets
//      that fall in the brick (counts, Eq. 5),
//   D. writes back the chunks whose codes changed as masks, and for chunks
//      with shadow counts c updates h' = min(h + c, H_max), sign 0 when
//      h < T <= h' (Eq. 6).
// AND is commutative and the saturating count with a threshold crossing
// depends only on the total count, so D gives exactly the state of applying
// the returns one by one in scan order (the first-return rule is resolved
// before this kernel).
#include "dbt_internal.cuh"

namespace dbt {

constexpr int WPC = 8;  // warps per CTA

struct WarpArea {
    uint32_t kst[BROWS * 8];  // codes: word kword(row, w) holds voxels x = 4w .. 4w+3 of a row
    uint16_t cnt[BVOX];       // shadow counts, index row * 32 + x
    uint8_t dirty[BROWS * 8]; // word changed (same index as kst)
    uint8_t need[BROWS];      // covered chunks of each row (bit w)
};
static_assert(sizeof(WarpArea) % 16 == 0, "warp area alignment");

// Word w of brick row `row`, with bit 2 of w flipped on rows 4-7 of each
// plane so that the 8-row x 4-word lane pattern of phase C is conflict-free.
__device__ __forceinline__ int kword(int row, int w) { return row * 8 + (w ^ (row & 4)); }

// Byte-wise unsigned minimum of four codes.
__device__ __forceinline__ uint32_t vmin4(uint32_t a, uint32_t b) { return __vminu4(a, b); }

__device__ __forceinline__ uint32_t code_to_mask(uint32_t k) {
    return k == 0u ? 0u : (0xFFFFFFFFu >> (32u - k));
}

template <int WL>
__global__ void __launch_bounds__(WPC * 32) k_integrate(DevGrid g, DevParams p, DevTables t,
                                                        long long n_input, WsDev ws) {
    extern __shared__ __align__(16) uint32_t smem[];
    constexpr int LY = 32 / WL;  // rows per lane group
    const int R = p.R;
    const int W = 2 * R + 4;
    const int np = (2 * R * R + 1) * W;
    uint32_t *P = smem;
    for (int j = threadIdx.x; j < np; j += blockDim.x) P[j] = t.prow[j];
    WarpArea *wa = reinterpret_cast<WarpArea *>(smem + ((np + 3) & ~3)) + (threadIdx.x >> 5);
    __syncthreads();

    const int lane = threadIdx.x & 31;
    const uint32_t nt = min(*(volatile uint32_t *)&ws.hdr->n_touched, ws.max_touched);
    const int SR = p.sr;
    const uint32_t T = (uint32_t)p.T, Hmax = (uint32_t)p.Hmax;

    for (;;) {
        uint32_t w = 0;
        if (lane == 0) w = atomicAdd(&ws.hdr->next_work, 1u);
        w = __shfl_sync(0xffffffffu, w, 0);
        if (w >= nt) break;
        const uint32_t b = ws.touched[w];
        const uint32_t start = ws.boff[b];
        uint32_t len = ws.bcnt[b];
        if ((unsigned long long)start + len > ws.pairs_cap) {  // cannot happen by sizing
            if (lane == 0) atomicOr(&ws.hdr->err, ERR_PAIRS_OVERFLOW);
            len = 0;
        }
        const int bx = (int)(b % (uint32_t)g.nbx);
        const uint32_t byz = b / (uint32_t)g.nbx;
        const int by = (int)(byz % (uint32_t)g.nby);
        const int bz = (int)(byz / (uint32_t)g.nby);
        const uint32_t *pairs = ws.pairs + start;

        // ---- A: covered chunks; lane owns rows `lane` and `lane + 32`
        {
            uint32_t need0 = 0, need1 = 0;
            const int ry = lane & 7, rz0 = lane >> 3, rz1 = rz0 + 4;
            for (uint32_t base = 0; base < len; base += 32) {
                const uint32_t mine = base + lane < len ? __ldg(pairs + base + lane) : 0u;
                const int cnt = (int)min(32u, len - base);
                for (int j = 0; j < cnt; ++j) {
                    const uint32_t pl = __shfl_sync(0xffffffffu, mine, j);
                    const int cx = (int)(pl & 63u) - R;
                    const int cy = (int)((pl >> 6) & 31u) - R;
                    const int cz = (int)((pl >> 11) & 31u) - R;
                    const int x0 = max(cx - R, 0), x1 = min(cx + R, BX - 1);
                    const uint32_t cm = (0xFFu >> (7 - (x1 >> 2))) & (0xFFu << (x0 >> 2));
                    const bool iny = ry >= cy - R && ry <= cy + R;
                    if (iny && rz0 >= cz - R && rz0 <= cz + R) need0 |= cm;
                    if (iny && rz1 >= cz - R && rz1 <= cz + R) need1 |= cm;
                }
            }
            wa->need[lane] = (uint8_t)need0;
            wa->need[lane + 32] = (uint8_t)need1;
        }
        __syncwarp();

        // ---- B: stage covered chunks as codes; lanes = 4 rows x 8 chunks
        const int rs = lane >> 3, ch = lane & 7;
        uint32_t form_bad = 0;
#pragma unroll 4
        for (int i = 0; i < 16; ++i) {
            const int row = rs + 4 * i;
            if ((wa->need[row] >> ch) & 1u) {
                const int gy = by * BY + (row & 7), gz = bz * BZ + (row >> 3);
                const size_t gi = ((size_t)gz * g.ny + gy) * g.pitch + (size_t)bx * BX + ch * 4;
                const uint4 m = __ldcg(reinterpret_cast<const uint4 *>(g.mask + gi));
                form_bad |= (m.x & (m.x + 1u)) | (m.y & (m.y + 1u)) | (m.z & (m.z + 1u)) |
                            (m.w & (m.w + 1u));
                const uint32_t k = (uint32_t)__popc(m.x) | ((uint32_t)__popc(m.y) << 8) |
                                   ((uint32_t)__popc(m.z) << 16) | ((uint32_t)__popc(m.w) << 24);
                wa->kst[kword(row, ch)] = k;
                wa->dirty[kword(row, ch)] = 0;
                *reinterpret_cast<uint2 *>(&wa->cnt[row * 32 + ch * 4]) = make_uint2(0u, 0u);
            }
        }
        if (form_bad) atomicOr(&ws.hdr->err, ERR_MASK_FORM);
        __syncwarp();

        // ---- C: Eqs. 4-5 on the staged brick
        const int ly = lane / WL, lw = lane % WL;
        for (uint32_t base = 0; base < len; base += 32) {
            const uint32_t mine = base + lane < len ? __ldg(pairs + base + lane) : 0u;
            const int cnt = (int)min(32u, len - base);
            for (int j = 0; j < cnt; ++j) {
                const uint32_t pl = __shfl_sync(0xffffffffu, mine, j);
                const int cx = (int)(pl & 63u) - R;
                const int cy = (int)((pl >> 6) & 31u) - R;
                const int cz = (int)((pl >> 11) & 31u) - R;
                const int x0 = max(cx - R, 0), x1 = min(cx + R, BX - 1);
                const int y0 = max(cy - R, 0), y1 = min(cy + R, BY - 1);
                const int z0 = max(cz - R, 0), z1 = min(cz + R, BZ - 1);
                const int wv = (x0 >> 2) + lw;
                const bool actw = wv <= (x1 >> 2);
                const int s = 4 * wv - cx + R + 3;
                for (int yb = y0; yb <= y1; yb += LY) {
                    const int ry = yb + ly;
                    const bool act = actw && ry <= y1;
                    const int oy = ry - cy;
                    const int pidx = oy * oy * W + s;
                    const int addr = ry * 8 + (wv ^ (ry & 4));
                    for (int rz = z0; rz <= z1; ++rz) {
                        const int oz = rz - cz;
                        if (act) {
                            const uint32_t kw = P[pidx + oz * oz * W];
                            uint32_t *cell = &wa->kst[rz * 64 + addr];
                            const uint32_t a = *cell;
                            const uint32_t nv = vmin4(a, kw);
                            if (nv != a) {
                                *cell = nv;
                                wa->dirty[rz * 64 + addr] = 1;
                            }
                        }
                    }
                }
                if (cx >= -SR && cx <= BX - 1 + SR && cy >= -SR && cy <= BY - 1 + SR &&
                    cz >= -SR && cz <= BZ - 1 + SR) {
                    const uint32_t bin = pl >> 16;
                    const uint32_t s1 = __ldg(&t.sh_start[bin + 1]);
                    for (uint32_t e = __ldg(&t.sh_start[bin]) + lane; e < s1; e += 32) {
                        const uint32_t o = __ldg(&t.sh_off[e]);
                        const int vx = cx + (int)(o & 255u) - 128;
                        const int vy = cy + (int)((o >> 8) & 255u) - 128;
                        const int vz = cz + (int)((o >> 16) & 255u) - 128;
                        if ((unsigned)vx < (unsigned)BX && (unsigned)vy < (unsigned)BY &&
                            (unsigned)vz < (unsigned)BZ)
                            wa->cnt[(vz * BY + vy) * BX + vx] += 1;
                    }
                }
                __syncwarp();
            }
        }

        // ---- D: write back
#pragma unroll 4
        for (int i = 0; i < 16; ++i) {
            const int row = rs + 4 * i;
            if ((wa->need[row] >> ch) & 1u) {
                const int gy = by * BY + (row & 7), gz = bz * BZ + (row >> 3);
                const size_t gi = ((size_t)gz * g.ny + gy) * g.pitch + (size_t)bx * BX + ch * 4;
                if (wa->dirty[kword(row, ch)]) {
                    const uint32_t k = wa->kst[kword(row, ch)];
                    const uint4 m = make_uint4(code_to_mask(k & 255u), code_to_mask((k >> 8) & 255u),
                                               code_to_mask((k >> 16) & 255u), code_to_mask(k >> 24));
                    __stcg(reinterpret_cast<uint4 *>(g.mask + gi), m);
                }
                const uint2 c = *reinterpret_cast<const uint2 *>(&wa->cnt[row * 32 + ch * 4]);
                if (c.x | c.y) {
                    uint2 hv = __ldcg(reinterpret_cast<const uint2 *>(g.hits + gi));
                    uint32_t sv = __ldcg(reinterpret_cast<const unsigned int *>(g.sign + gi));
                    const uint32_t cnt4[4] = {c.x & 0xFFFFu, c.x >> 16, c.y & 0xFFFFu, c.y >> 16};
                    uint32_t h[4] = {hv.x & 0xFFFFu, hv.x >> 16, hv.y & 0xFFFFu, hv.y >> 16};
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        if (cnt4[e]) {
                            const uint32_t ho = h[e];
                            const uint32_t hn = min(ho + cnt4[e], Hmax);
                            if (ho < T && hn >= T) sv &= ~(0xFFu << (8 * e));
                            h[e] = hn;
                        }
                    }
                    hv.x = h[0] | (h[1] << 16);
                    hv.y = h[2] | (h[3] << 16);
                    __stcg(reinterpret_cast<uint2 *>(g.hits + gi), hv);
                    __stcg(reinterpret_cast<unsigned int *>(g.sign + gi), sv);
                }
            }
        }
        if (lane == 0) ws.bcnt[b] = 0u;
        __syncwarp();
    }

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
            h->err = 0u;
            h->n_touched = 0u;
            h->pool = 0u;
            h->next_work = 0u;
            h->acc_valid = 0ull;
            h->acc_inside = 0ull;
            h->acc_kept = 0ull;
            __threadfence();
            h->done_ctas = 0u;
        }
    }
}

// Dynamic shared memory of one CTA for kernel size K.
static size_t integrate_smem(int K) {
    const int R = (K - 1) / 2;
    const size_t np = (size_t)(2 * R * R + 1) * (2 * R + 4);
    return ((np + 3) & ~size_t(3)) * 4 + WPC * sizeof(WarpArea);
}

struct IntegrateCfg {
    int device = -1;
    int ctas[MAX_K + 1] = {};
};
static IntegrateCfg g_cfg;

// Occupancy-based persistent grid for one kernel size; the shared-memory
// limit of each template instance is raised once per device to what its
// largest kernel size needs (the attribute belongs to the function, so it
// must not be lowered for a smaller K).
template <int WL>
static int configure(size_t smem, size_t smem_max) {
    static int limit_set_on = -1;
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    if (limit_set_on != dev) {
        cudaFuncSetAttribute(k_integrate<WL>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem_max);
        limit_set_on = dev;
    }
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_integrate<WL>, WPC * 32, smem);
    return max(1, sms * max(1, per_sm));
}

// Persistent grid for kernel size K: every SM filled to its occupancy limit.
int integrate_grid_ctas(int K) {
    int dev = 0;
    cudaGetDevice(&dev);
    if (g_cfg.device != dev) {
        g_cfg = IntegrateCfg();
        g_cfg.device = dev;
    }
    if (!g_cfg.ctas[K]) {
        const size_t smem = integrate_smem(K);
        g_cfg.ctas[K] = K <= 13 ? configure<4>(smem, integrate_smem(13))
                                : configure<8>(smem, integrate_smem(MAX_K));
    }
    return g_cfg.ctas[K];
}

void launch_integrate(const DevGrid &g, const DevParams &p, const DevTables &t, long long n_input,
                      const WsDev &ws, int grid_ctas, cudaStream_t s) {
    const size_t smem = integrate_smem(p.K);
    if (p.K <= 13)
        k_integrate<4><<<grid_ctas, WPC * 32, smem, s>>>(g, p, t, n_input, ws);
    else
        k_integrate<8><<<grid_ctas, WPC * 32, smem, s>>>(g, p, t, n_input, ws);
}

}  // namespace dbt
