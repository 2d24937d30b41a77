/*
 * Points-parallel variant of the DB-TSDF oracle -- TEST AND BASELINE
 * INFRASTRUCTURE ONLY.  Only tests/ and the CPU baseline leg of bench.py load
 * it; the product path never does.
 *
 * The paper runs its per-return updates in parallel over the returns on the
 * host cores (OpenMP, Sec. IV).  This file does the same on top of the
 * oracle's own definitions: dbtsdf_oracle.c is compiled into this library
 * (included below), so every step -- transform, contact voxel, bin (Sec.
 * III-C), kernel mask (Eq. 3), shadow set (Sec. III-B) -- is the oracle's
 * function.  Per scan:
 *   1. every return's contact and bin, in parallel (orc_contact);
 *   2. the first-return rule of Sec. IV-B in array order (sequential);
 *   3. the Eq. 4-6 updates of the kept returns in parallel, each voxel
 *      changed by an atomic operation.
 * The kernel masks and the bins' shadow sets are tabulated once per call, as
 * the paper precomputes its directional kernels.
 *
 * Exact: AND is commutative, a saturating counter bumped c times ends at
 * min(h + c, H_max) in any order, and with 1 <= T <= H_max exactly one bump
 * takes it from T - 1 to T -- the one that sets the sign to occupied (the
 * sign only ever goes that way).  So the map equals the sequential oracle's
 * bit for bit (tests/test_oracle_omp.py), unlike an update without atomics,
 * where two threads can lose each other's writes.  n_mask_writes is the one
 * counter that depends on the order (which write of a voxel changes it); the
 * other counters are the sequential oracle's.
 */
#include "dbtsdf_oracle.c"

#include <omp.h>

int orc_omp_max_threads(void) { return omp_get_max_threads(); }

int64_t orc_integrate_scan_omp(orc_grid *g, const orc_params *p, const float *xyz, int64_t n,
                               const double pose[12], int threads, orc_stats *st_out)
{
    orc_stats st;
    memset(&st, 0, sizeof st);
    if (p->kernel_size < 1 || (p->kernel_size & 1) == 0 || n < 0 || threads < 1)
        return -1;
    const int K = p->kernel_size, R = (K - 1) / 2;
    const int64_t K3 = (int64_t)K * K * K;
    const int nb = orc_num_bins(p);
    const int64_t nv = g->nx * g->ny * g->nz;
    const int64_t nn = n > 0 ? n : 1;
    int64_t *c = (int64_t *)malloc((size_t)nn * 3 * sizeof(int64_t));
    int32_t *b = (int32_t *)malloc((size_t)nn * sizeof(int32_t));
    uint8_t *in = (uint8_t *)malloc((size_t)nn);
    uint32_t *kmask = (uint32_t *)malloc((size_t)K3 * sizeof(uint32_t));
    uint8_t *shadow = (uint8_t *)malloc((size_t)nb * (size_t)K3);
    uint8_t *seen = p->dedup_first ? (uint8_t *)calloc((size_t)((nv + 7) / 8), 1) : NULL;
    int fail = !c || !b || !in || !kmask || !shadow || (p->dedup_first && !seen);
    if (fail)
        goto out;

    /* Eq. 3 masks and the shadow sets S_b over the kernel, [oz][oy][ox] */
    for (int oz = -R; oz <= R; oz++)
        for (int oy = -R; oy <= R; oy++)
            for (int ox = -R; ox <= R; ox++)
                kmask[((oz + R) * K + (oy + R)) * K + (ox + R)] = orc_distance_mask(ox, oy, oz);
#pragma omp parallel for num_threads(threads) schedule(static)
    for (int bb = 0; bb < nb; bb++)
        for (int oz = -R; oz <= R; oz++)
            for (int oy = -R; oy <= R; oy++)
                for (int ox = -R; ox <= R; ox++)
                    shadow[(int64_t)bb * K3 + ((oz + R) * K + (oy + R)) * K + (ox + R)] =
                        (uint8_t)orc_in_shadow(p, bb, ox, oy, oz);

    /* 1. contacts and bins of every return */
    int64_t n_valid = 0, n_inside = 0;
#pragma omp parallel for num_threads(threads) schedule(static) reduction(+ : n_valid, n_inside)
    for (int64_t i = 0; i < n; i++) {
        int bin = 0, valid = 0;
        in[i] = (uint8_t)orc_contact(p, g, xyz + 3 * i, pose, c + 3 * i, &bin, &valid);
        b[i] = bin;
        n_valid += valid;
        n_inside += in[i];
    }
    st.n_input = n;
    st.n_valid = n_valid;
    st.n_inside = n_inside;

    /* 2. first return per contact voxel, in array order; kept returns are
     * compacted to the front of c and b */
    int64_t m = 0;
    for (int64_t i = 0; i < n; i++) {
        if (!in[i])
            continue;
        if (seen) {
            int64_t v = (c[3 * i + 2] * g->ny + c[3 * i + 1]) * g->nx + c[3 * i + 0];
            if (seen[v >> 3] & (1u << (v & 7)))
                continue;
            seen[v >> 3] |= (uint8_t)(1u << (v & 7));
        }
        c[3 * m + 0] = c[3 * i + 0];
        c[3 * m + 1] = c[3 * i + 1];
        c[3 * m + 2] = c[3 * i + 2];
        b[m] = b[i];
        m++;
    }
    st.n_kept = m;

    /* 3. Eqs. 4-6 of the kept returns, one atomic operation per voxel field */
    int64_t writes = 0, incs = 0;
    const int T = p->hit_threshold, Hmax = p->hit_max;
#pragma omp parallel for num_threads(threads) schedule(dynamic, 16) reduction(+ : writes, incs)
    for (int64_t j = 0; j < m; j++) {
        const uint8_t *sh = shadow + (int64_t)b[j] * K3;
        int64_t t = 0;
        for (int oz = -R; oz <= R; oz++)
            for (int oy = -R; oy <= R; oy++) {
                const int64_t row = ((c[3 * j + 2] + oz) * g->ny + (c[3 * j + 1] + oy)) * g->nx +
                                    c[3 * j + 0];
                for (int ox = -R; ox <= R; ox++, t++) {
                    const int64_t v = row + ox;
                    const uint32_t k = kmask[t];
                    const uint32_t cur = __atomic_load_n(&g->mask[v], __ATOMIC_RELAXED);
                    if ((cur & k) != cur) {                                   /* Eq. 4 */
                        const uint32_t old = __atomic_fetch_and(&g->mask[v], k, __ATOMIC_RELAXED);
                        writes += (old & k) != old;
                    }
                    if (sh[t]) {
                        uint16_t h_old = __atomic_load_n(&g->hits[v], __ATOMIC_RELAXED);
                        uint16_t h_new;
                        do {                                                  /* Eq. 5 */
                            h_new = (uint16_t)(h_old + 1 > Hmax ? Hmax : h_old + 1);
                        } while (!__atomic_compare_exchange_n(&g->hits[v], &h_old, h_new, 1,
                                                              __ATOMIC_RELAXED, __ATOMIC_RELAXED));
                        if (h_old < T && h_new >= T)                          /* Eq. 6 */
                            __atomic_store_n(&g->sign[v], (uint8_t)0, __ATOMIC_RELAXED);
                        incs++;
                    }
                }
            }
    }
    st.n_mask_writes = writes;
    st.n_shadow_incs = incs;

out:
    free(c);
    free(b);
    free(in);
    free(kmask);
    free(shadow);
    free(seen);
    if (fail)
        return -1;
    if (st_out)
        *st_out = st;
    return st.n_kept;
}
