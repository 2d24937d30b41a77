// Brick integration of one scan (Sec. III-C, Eqs. 4-6).
//
// A persistent CTA takes touched bricks (32 x 8 x 8 voxels) from a dynamic
// queue.  For each brick it
//   A. marks which 16-byte chunks of the brick's 64 rows any of its returns'
//      K^3 neighbourhoods cover (one 8-bit chunk mask per row),
//   B. stages exactly those chunks of the mask plane in shared memory and
//      zeroes a shared 32-bit shadow counter per staged voxel,
//   C. applies every (return, brick) pair: the kernel's Eq. 3 masks are ANDed
//      into the staged masks (read first, atomicAnd only when a bit clears,
//      the skip of Eq. 4), and each voxel of the bin's hemispherical shadow
//      gets a shared atomicAdd,
//   D. writes back the chunks whose masks changed, and for chunks with shadow
//      hits updates the hit counter and sign once per voxel:
//      h' = min(h + c, H_max), sign -> 0 when h < T <= h'.
// Because AND is commutative and the saturating count with a threshold
// crossing depends only on the total, D gives exactly the state of applying
// the returns one by one in scan order (the first-return rule is resolved
// before this kernel).  Rows alternate a 16-word XOR swizzle so that the two
// half-warps working on neighbouring rows hit different banks.
#include "dbt_internal.cuh"

namespace dbt {

__device__ __forceinline__ int swz(int row, int x) { return row * BX + (x ^ ((row & 1) << 4)); }

template <int LX>
__global__ void __launch_bounds__(256) k_integrate(DevGrid g, DevParams p, DevTables t,
                                                   long long n_input, WsDev ws) {
    constexpr int ROWS_PER_IT = 32 / LX;
    __shared__ __align__(16) uint32_t s_mask[BVOX];
    __shared__ __align__(16) uint32_t s_cnt[BVOX];
    __shared__ uint32_t s_need[BROWS];
    __shared__ uint32_t s_m2[MAX_M2];
    __shared__ uint32_t s_work;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nwarps = blockDim.x >> 5;
    const int R = p.R;
    for (int j = tid; j < p.n_m2; j += blockDim.x) s_m2[j] = t.m2[j];
    const uint32_t nt = min(*(volatile uint32_t *)&ws.hdr->n_touched, ws.max_touched);

    for (;;) {
        __syncthreads();
        if (tid == 0) s_work = atomicAdd(&ws.hdr->next_work, 1u);
        if (tid < BROWS) s_need[tid] = 0u;
        __syncthreads();
        const uint32_t w = s_work;
        if (w >= nt) break;
        const uint32_t b = ws.touched[w];
        const uint32_t start = ws.boff[b];
        uint32_t len = ws.bcnt[b];
        if ((unsigned long long)start + len > ws.pairs_cap) {   // cannot happen by sizing
            if (tid == 0) atomicOr(&ws.hdr->err, ERR_PAIRS_OVERFLOW);
            len = 0;
        }
        const int bx = (int)(b % (uint32_t)g.nbx);
        const uint32_t byz = b / (uint32_t)g.nbx;
        const int by = (int)(byz % (uint32_t)g.nby);
        const int bz = (int)(byz / (uint32_t)g.nby);

        // ---- A: chunk coverage
        for (uint32_t j = warp; j < len; j += nwarps) {
            const uint32_t pl = ws.pairs[start + j];
            const int cx = (int)(pl & 63u) - R;
            const int cy = (int)((pl >> 6) & 31u) - R;
            const int cz = (int)((pl >> 11) & 31u) - R;
            const int x0 = max(cx - R, 0), x1 = min(cx + R, BX - 1);
            const int y0 = max(cy - R, 0), y1 = min(cy + R, BY - 1);
            const int z0 = max(cz - R, 0), z1 = min(cz + R, BZ - 1);
            const uint32_t cm = (0xFFu >> (7 - (x1 >> 2))) & (0xFFu << (x0 >> 2));
            const int wy = y1 - y0 + 1;
            const int nrows = wy * (z1 - z0 + 1);
            for (int r = lane; r < nrows; r += 32) {
                const int q = r / wy;
                atomicOr(&s_need[(z0 + q) * BY + y0 + (r - q * wy)], cm);
            }
        }
        __syncthreads();

        // ---- B: stage the covered chunks
        uint4 orig[BCHUNKS / 256];
#pragma unroll
        for (int k = 0; k < BCHUNKS / 256; ++k) {
            const int c = tid + k * 256;
            const int row = c >> 3, ch = c & 7;
            orig[k] = make_uint4(0, 0, 0, 0);
            if ((s_need[row] >> ch) & 1u) {
                const int gy = by * BY + (row & (BY - 1));
                const int gz = bz * BZ + row / BY;
                const size_t gi = ((size_t)gz * g.ny + gy) * g.pitch + (size_t)bx * BX + ch * 4;
                const uint4 v = __ldcg(reinterpret_cast<const uint4 *>(g.mask + gi));
                orig[k] = v;
                const int a = swz(row, ch * 4);
                *reinterpret_cast<uint4 *>(&s_mask[a]) = v;
                *reinterpret_cast<uint4 *>(&s_cnt[a]) = make_uint4(0, 0, 0, 0);
            }
        }
        __syncthreads();

        // ---- C: Eqs. 4-5 in shared memory
        const int xi = lane % LX;
        const int half = lane / LX;
        for (uint32_t j = warp; j < len; j += nwarps) {
            const uint32_t pl = ws.pairs[start + j];
            const int cx = (int)(pl & 63u) - R;
            const int cy = (int)((pl >> 6) & 31u) - R;
            const int cz = (int)((pl >> 11) & 31u) - R;
            const uint32_t bin = pl >> 16;
            const int x0 = max(cx - R, 0), x1 = min(cx + R, BX - 1);
            const int y0 = max(cy - R, 0), y1 = min(cy + R, BY - 1);
            const int z0 = max(cz - R, 0), z1 = min(cz + R, BZ - 1);
            const int wy = y1 - y0 + 1;
            const int x = x0 + xi;
            const bool xon = x <= x1;
            const int ox = x - cx;
            const int oxsq = ox * ox;
            int ry = y0 + half, rz = z0;
            while (ry > y1) { ry -= wy; ++rz; }
            while (rz <= z1) {
                if (xon) {
                    const int oy = ry - cy, oz = rz - cz;
                    const uint32_t m = s_m2[oxsq + oy * oy + oz * oz];
                    const int a = swz(rz * BY + ry, x);
                    const uint32_t old = s_mask[a];
                    if ((old & m) != old) atomicAnd(&s_mask[a], m);
                }
                ry += ROWS_PER_IT;
                while (ry > y1) { ry -= wy; ++rz; }
            }
            const uint32_t s0 = __ldg(&t.sh_start[bin]);
            const uint32_t s1 = __ldg(&t.sh_start[bin + 1]);
            for (uint32_t e = s0 + lane; e < s1; e += 32) {
                const uint32_t o = __ldg(&t.sh_off[e]);
                const int vx = cx + (int)(o & 255u) - 128;
                const int vy = cy + (int)((o >> 8) & 255u) - 128;
                const int vz = cz + (int)((o >> 16) & 255u) - 128;
                if ((unsigned)vx < (unsigned)BX && (unsigned)vy < (unsigned)BY &&
                    (unsigned)vz < (unsigned)BZ)
                    atomicAdd(&s_cnt[swz(vz * BY + vy, vx)], 1u);
            }
        }
        __syncthreads();

        // ---- D: write back
#pragma unroll
        for (int k = 0; k < BCHUNKS / 256; ++k) {
            const int c = tid + k * 256;
            const int row = c >> 3, ch = c & 7;
            if ((s_need[row] >> ch) & 1u) {
                const int gy = by * BY + (row & (BY - 1));
                const int gz = bz * BZ + row / BY;
                const size_t gi = ((size_t)gz * g.ny + gy) * g.pitch + (size_t)bx * BX + ch * 4;
                const int a = swz(row, ch * 4);
                const uint4 nv = *reinterpret_cast<const uint4 *>(&s_mask[a]);
                if (nv.x != orig[k].x || nv.y != orig[k].y || nv.z != orig[k].z || nv.w != orig[k].w)
                    __stcg(reinterpret_cast<uint4 *>(g.mask + gi), nv);
                const uint4 cv = *reinterpret_cast<const uint4 *>(&s_cnt[a]);
                if (cv.x | cv.y | cv.z | cv.w) {
                    uint2 hv = __ldcg(reinterpret_cast<const uint2 *>(g.hits + gi));
                    uint32_t sv = __ldcg(reinterpret_cast<const unsigned int *>(g.sign + gi));
                    const uint32_t cnt[4] = {cv.x, cv.y, cv.z, cv.w};
                    uint32_t h[4] = {hv.x & 0xFFFFu, hv.x >> 16, hv.y & 0xFFFFu, hv.y >> 16};
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        if (cnt[e]) {
                            const uint32_t ho = h[e];
                            const uint32_t hn = min(ho + cnt[e], (uint32_t)p.Hmax);
                            if (ho < (uint32_t)p.T && hn >= (uint32_t)p.T) sv &= ~(0xFFu << (8 * e));
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
        if (tid == 0) ws.bcnt[b] = 0u;
    }

    // Last CTA out publishes the scan's counters and re-arms the workspace.
    __syncthreads();
    if (tid == 0) {
        __threadfence();
        if (atomicAdd(&ws.hdr->done_ctas, 1u) == gridDim.x - 1) {
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

static int g_integrate_ctas[2] = {0, 0};

static int occupancy_ctas(int lx) {
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (lx == 16)
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_integrate<16>, 256, 0);
    else
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_integrate<32>, 256, 0);
    return max(1, sms * max(1, per_sm));
}

// Persistent grid: every SM filled to its occupancy limit.
int integrate_grid_ctas(int K) {
    const int v = K <= 16 ? 0 : 1;
    if (!g_integrate_ctas[v]) g_integrate_ctas[v] = occupancy_ctas(v == 0 ? 16 : 32);
    return g_integrate_ctas[v];
}

void launch_integrate(const DevGrid &g, const DevParams &p, const DevTables &t, long long n_input,
                      const WsDev &ws, int grid_ctas, cudaStream_t s) {
    if (p.K <= 16) {
        k_integrate<16><<<grid_ctas, 256, 0, s>>>(g, p, t, n_input, ws);
    } else {
        k_integrate<32><<<grid_ctas, 256, 0, s>>>(g, p, t, n_input, ws);
    }
}

}  // namespace dbt
