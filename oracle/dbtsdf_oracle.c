/*
 * DB-TSDF reference integrator (the oracle) -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, single-threaded C restatement of the scan integration of
 * DB-TSDF (arXiv 2509.20081, Sec. III).  It exists so that the CUDA library
 * can be checked voxel by voxel.  Only tests/, the smoke check and the CPU
 * baseline leg of bench.py may load it; the product path never does.  It
 * shares no code, header, table or constant with the CUDA library.
 *
 * Floating point: every step that turns a float into an integer (voxel index,
 * direction bin) is evaluated in IEEE binary64 with basic operations only
 * (each rounded to nearest), in the order written here; this file must be
 * compiled with -ffp-contract=off so that no multiply-add is fused.  The
 * paper writes the steps as formulas (Sec. III-C: p_w = R p + t, voxel index
 * floor((p_w - o) / res)); they are evaluated as written:
 *   d = R p with each row as (r0 * x + r1 * y) + r2 * z; w = d + t;
 *   c = floor((w - origin) / res), a true division;
 *   octahedral u = d_x / s, v = d_y / s, s = (|x| + |y|) + |z|.
 *
 * Readings of the paper taken where it is silent or ambiguous (each is listed
 * with its reason in the design notes of the repository):
 *   - Eq. 3 uses the Euclidean r and ceil(r) bits (not the "L1" of Sec. III-A).
 *   - a return is discarded when a coordinate is not finite, when it is the
 *     origin, or when its K^3 neighbourhood leaves the grid (Sec. III-C):
 *     kept iff R <= c_i <= N_i - 1 - R on every axis.
 *   - the direction that selects the bin is the map-frame ray d = R p.
 *   - Eq. 2 azimuth is taken modulo 2 pi, the elevation bin is clamped to
 *     B_el - 1, and both are decided by comparing against the bin edges
 *     (ties go to the higher bin) instead of calling atan2/asin.
 *   - octahedral bins (not in the paper) follow the octahedral map.
 *   - the shadow set S_b = { o : |o|^2 <= r_s^2 and o . u_b >= 0 }, plane and
 *     centre included, sign of o . u_b decided exactly.
 *   - "only the first is integrated" (Sec. IV-B): first = lowest array index
 *     among returns that survived the discards, per contact voxel, per scan.
 *   - Eq. 6 with h_new >= T; T and H_max are parameters with 1 <= T <= H_max.
 * Parity unpinned: the defaults of T, H_max and r_s (the paper gives none).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* pi rounded to the nearest binary64 value */
#define ORC_PI 3.14159265358979323846

#define ORC_SCHEME_OCTA 0
#define ORC_SCHEME_AZEL 1

typedef struct {
    int kernel_size;      /* K, odd; the neighbourhood is [-R, R]^3, R = (K-1)/2 */
    int scheme;           /* ORC_SCHEME_OCTA or ORC_SCHEME_AZEL */
    int bins_a;           /* octa: n (n x n cells); azel: B_az */
    int bins_b;           /* octa: n;               azel: B_el */
    double shadow_radius; /* r_s in voxels */
    int hit_threshold;    /* T */
    int hit_max;          /* H_max */
    int dedup_first;      /* 1: only the first return per contact voxel */
    double shadow_cos;    /* 0: hemispherical shadow; c > 0: cone, cos(half-angle) = c */
} orc_params;

typedef struct {
    int64_t nx, ny, nz;   /* voxels per axis; dense, x fastest, no padding */
    double res;           /* voxel edge in metres */
    double origin[3];     /* map-frame position of the corner of voxel (0,0,0) */
    uint32_t *mask;
    uint8_t *sign;
    uint16_t *hits;
} orc_grid;

typedef struct {
    int64_t n_input;      /* returns handed in */
    int64_t n_valid;      /* finite and not the origin */
    int64_t n_inside;     /* neighbourhood inside the map */
    int64_t n_kept;       /* integrated (after first-per-voxel) */
    int64_t n_mask_writes;/* Eq. 4 writes that changed a mask */
    int64_t n_shadow_incs;/* Eq. 5 applications (before saturation) */
} orc_stats;

/* ------------------------------------------------------------------ */
/* Sec. III-A: initial voxel state -- all mask bits set, sign free (1),
 * counter zero.                                                       */
void orc_grid_init(orc_grid *g)
{
    int64_t nv = g->nx * g->ny * g->nz;
    for (int64_t i = 0; i < nv; i++) {
        g->mask[i] = 0xFFFFFFFFu;
        g->sign[i] = 1;
        g->hits[i] = 0;
    }
}

/* Eq. 1: M_grid = Nx Ny Nz S_voxel, with the paper's S_voxel = 8 bytes. */
int64_t orc_grid_bytes_eq1(int64_t nx, int64_t ny, int64_t nz)
{
    return nx * ny * nz * 8;
}

/* ------------------------------------------------------------------ */
/* Eq. 3: m(x,y,z) = 0 when r = 0, else (2^32 - 1) >> (32 - ceil(r)),
 * r = sqrt(x^2 + y^2 + z^2) in voxel units.  For ceil(r) >= 32 no bit is
 * shifted out and the mask stays all ones.                            */
uint32_t orc_distance_mask(int x, int y, int z)
{
    double r = sqrt((double)x * x + (double)y * y + (double)z * z);
    if (r == 0.0)
        return 0u;
    int c = (int)ceil(r);
    if (c >= 32)
        return 0xFFFFFFFFu;
    return 0xFFFFFFFFu >> (32 - c);
}

/* ------------------------------------------------------------------ */
/* Direction bins.                                                       */

static double orc_sgn(double v) { return v < 0.0 ? -1.0 : 1.0; }

/* Octahedral bins (the workloads' 8x8 scheme; not in the paper).  The ray d is
 * projected on the octahedron |x|+|y|+|z| = 1; the lower half (z < 0) is
 * folded over the diagonals; the square [-1,1]^2 is cut into n x n cells.
 * Returns j * n + i for the cell (i along u, j along v).               */
int orc_bin_octa(double dx, double dy, double dz, int n)
{
    double s = (fabs(dx) + fabs(dy)) + fabs(dz);
    if (!(s > 0.0))
        return 0;                       /* no direction (not reached for a rotation) */
    double u = dx / s;
    double v = dy / s;
    if (dz < 0.0) {
        double fu = (1.0 - fabs(v)) * orc_sgn(u);
        double fv = (1.0 - fabs(u)) * orc_sgn(v);
        u = fu;
        v = fv;
    }
    int i = (int)floor(((u + 1.0) * 0.5) * (double)n);
    int j = (int)floor(((v + 1.0) * 0.5) * (double)n);
    if (i > n - 1) i = n - 1;
    if (j > n - 1) j = n - 1;
    if (i < 0) i = 0;
    if (j < 0) j = 0;
    return j * n + i;
}

/* Representative direction of octahedral cell b: the octahedral decode of
 * the cell centre, scaled by n so that every component is an integer (the
 * scale is positive, so the sign of o . u_b is unchanged).            */
void orc_bin_octa_dir(int b, int n, double out[3])
{
    int i = b % n, j = b / n;
    double U = (double)(2 * i + 1 - n);   /* n times the centre's u */
    double V = (double)(2 * j + 1 - n);
    double Z = (double)n - fabs(U) - fabs(V);
    if (Z < 0.0) {
        double fu = ((double)n - fabs(V)) * orc_sgn(U);
        double fv = ((double)n - fabs(U)) * orc_sgn(V);
        U = fu;
        V = fv;
    }
    out[0] = U;
    out[1] = V;
    out[2] = Z;
}

/* Bin edges of Eq. 2.  Azimuth edge k: theta_k = (2 pi k) / B_az; elevation
 * edge k: phi_k = (pi k) / B_el - pi / 2.                              */
static double orc_az_edge(int k, int baz) { return ((2.0 * ORC_PI) * (double)k) / (double)baz; }
static double orc_el_edge(int k, int bel) { return (ORC_PI * (double)k) / (double)bel - ORC_PI / 2.0; }

/* Eq. 2, azimuth: b_az = floor(theta / (2 pi) * B_az), theta = atan2(y, x)
 * taken in [0, 2 pi).  In exact arithmetic this is the number of edges
 * theta_k (k = 1 .. B_az-1) with theta >= theta_k.  For theta and theta_k
 * on the same side of the pi line (or theta_k < pi <= theta) the test is
 * the sign of sin(theta - theta_k) = cos(theta_k) y - sin(theta_k) x.   */
int orc_bin_az(double x, double y, int baz)
{
    if (x == 0.0 && y == 0.0)
        return 0;                                     /* atan2(0, 0) = 0 */
    int upper = (y > 0.0) || (y == 0.0 && x >= 0.0);  /* theta in [0, pi) */
    int b = 0;
    for (int k = 1; k < baz; k++) {
        double t = orc_az_edge(k, baz);
        int edge_upper = t < ORC_PI;
        int ge;
        if (upper && !edge_upper)
            ge = 0;                       /* theta < pi <= theta_k */
        else if (!upper && edge_upper)
            ge = 1;                       /* theta_k < pi <= theta */
        else
            ge = (cos(t) * y - sin(t) * x) >= 0.0;
        b += ge;
    }
    return b;
}

/* Eq. 2, elevation: b_el = floor((asin(z/|p|) + pi/2) / pi * B_el), clamped
 * to B_el - 1.  asin is increasing, so this counts the edges k = 1..B_el-1
 * with z/|p| >= sin(phi_k).                                            */
int orc_bin_el(double x, double y, double z, int bel)
{
    double norm = sqrt((x * x + y * y) + z * z);
    double s = z / norm;
    int b = 0;
    for (int k = 1; k < bel; k++)
        b += s >= sin(orc_el_edge(k, bel));
    return b;
}

/* Eq. 2 bin id, az-major: b = b_el * B_az + b_az.                      */
int orc_bin_azel(double x, double y, double z, int baz, int bel)
{
    return orc_bin_el(x, y, z, bel) * baz + orc_bin_az(x, y, baz);
}

/* Representative unit vector of az/el bin b: the centre of its azimuth
 * and elevation intervals (Sec. III-B).                                */
void orc_bin_azel_dir(int b, int baz, int bel, double out[3])
{
    int a = b % baz, e = b / baz;
    double alpha = ((2.0 * ORC_PI) * ((double)a + 0.5)) / (double)baz;
    double eps = (ORC_PI * ((double)e + 0.5)) / (double)bel - ORC_PI / 2.0;
    out[0] = cos(eps) * cos(alpha);
    out[1] = cos(eps) * sin(alpha);
    out[2] = sin(eps);
}

int orc_bin(const orc_params *p, double dx, double dy, double dz)
{
    if (p->scheme == ORC_SCHEME_OCTA)
        return orc_bin_octa(dx, dy, dz, p->bins_a);
    return orc_bin_azel(dx, dy, dz, p->bins_a, p->bins_b);
}

int orc_num_bins(const orc_params *p)
{
    return p->bins_a * p->bins_b;
}

void orc_bin_dir(const orc_params *p, int b, double out[3])
{
    if (p->scheme == ORC_SCHEME_OCTA)
        orc_bin_octa_dir(b, p->bins_a, out);
    else
        orc_bin_azel_dir(b, p->bins_a, p->bins_b, out);
}

/* ------------------------------------------------------------------ */
/* Sec. III-B: shadow set.  Offset o is in the shadow of bin b when its
 * centre lies in the Euclidean ball of radius r_s around the contact voxel
 * and not in the half facing the sensor, o . u_b >= 0 (the hemisphere).
 * The conical model of the same section (shadow_cos = c > 0) keeps, of that
 * ball, the offsets within the half-angle acos(c) of the bin direction:
 * o . u_b >= c |o| |u_b|.  u_b as returned by orc_bin_dir (not normalised
 * for the octahedral scheme, so the hemisphere test is exact there).     */
int orc_in_shadow(const orc_params *p, int b, int ox, int oy, int oz)
{
    double r2 = (double)ox * ox + (double)oy * oy + (double)oz * oz;
    if (!(r2 <= p->shadow_radius * p->shadow_radius))
        return 0;
    double u[3];
    orc_bin_dir(p, b, u);
    double dot = ((double)ox * u[0] + (double)oy * u[1]) + (double)oz * u[2];
    if (p->shadow_cos == 0.0)
        return dot >= 0.0;
    double uu = (u[0] * u[0] + u[1] * u[1]) + u[2] * u[2];
    return dot >= p->shadow_cos * sqrt(r2 * uu);
}

/* ------------------------------------------------------------------ */
/* Sec. III-C, first steps for one return: map-frame transform with the pose
 * (row-major 3x4 [R | t]), voxel of contact, boundary discard and bin.
 * Returns 0 when the return is discarded.                              */
int orc_contact(const orc_params *p, const orc_grid *g, const float *xyz,
                const double pose[12], int64_t c[3], int *bin, int *valid)
{
    double px = xyz[0], py = xyz[1], pz = xyz[2];
    *valid = 0;
    if (!isfinite(px) || !isfinite(py) || !isfinite(pz))
        return 0;
    if (px == 0.0 && py == 0.0 && pz == 0.0)
        return 0;
    *valid = 1;
    double d[3], w[3];
    for (int r = 0; r < 3; r++) {
        d[r] = (pose[4 * r + 0] * px + pose[4 * r + 1] * py) + pose[4 * r + 2] * pz;
        w[r] = d[r] + pose[4 * r + 3];
    }
    int R = (p->kernel_size - 1) / 2;
    int64_t n[3] = {g->nx, g->ny, g->nz};
    for (int a = 0; a < 3; a++) {
        double q = floor((w[a] - g->origin[a]) / g->res);
        if (!(q >= (double)R && q <= (double)(n[a] - 1 - R)))
            return 0;
        c[a] = (int64_t)q;
    }
    *bin = orc_bin(p, d[0], d[1], d[2]);
    return 1;
}

/* Eqs. 4-6 for one kept return with contact voxel c and bin b: every voxel
 * of the K^3 neighbourhood gets its mask ANDed with the kernel mask (the
 * write skipped when nothing changes); voxels of the shadow set get their
 * saturating counter bumped and their sign set to occupied when the counter
 * crosses T.                                                            */
static void orc_apply_kernel(orc_grid *g, const orc_params *p, const int64_t c[3], int b,
                             orc_stats *st)
{
    int R = (p->kernel_size - 1) / 2;
    for (int oz = -R; oz <= R; oz++)
        for (int oy = -R; oy <= R; oy++)
            for (int ox = -R; ox <= R; ox++) {
                int64_t v = ((c[2] + oz) * g->ny + (c[1] + oy)) * g->nx + (c[0] + ox);
                uint32_t m = g->mask[v];
                uint32_t k = orc_distance_mask(ox, oy, oz);
                if (m != (m & k)) {                          /* Eq. 4 */
                    g->mask[v] = m & k;
                    st->n_mask_writes++;
                }
                if (orc_in_shadow(p, b, ox, oy, oz)) {
                    int h_old = g->hits[v];
                    int h_new = h_old + 1;                   /* Eq. 5 */
                    if (h_new > p->hit_max)
                        h_new = p->hit_max;
                    g->hits[v] = (uint16_t)h_new;
                    if (h_old < p->hit_threshold && h_new >= p->hit_threshold)
                        g->sign[v] = 0;                      /* Eq. 6 */
                    st->n_shadow_incs++;
                }
            }
}

/* One scan, returns in array order (Sec. III-C with the first-return rule
 * of Sec. IV-B).  Returns the number of kept returns, or -1 on a bad
 * argument or an allocation failure.                                   */
/* Sec. III-C with the update's optional pre-steps:
 *   - sequential downsampling (Sec. IV-B, "DS"): only returns whose index is
 *     a multiple of ds are handed to the update (ds = 1: all);
 *   - motion compensation (Sec. III-C, Fig. 3): return i is transformed with
 *     its own pose poses[m(i)], m(i) = ((i mod period) * n_poses) / period,
 *     i.e. the sweep's time runs with the index modulo period (period = the
 *     returns per beam of a beam-major spinning scan, or n for returns in
 *     acquisition order) and is cut into n_poses equal slices.
 * n_poses = 1 is the single-pose update.  Returns the kept count or -1.    */
int64_t orc_integrate_scan_ex(orc_grid *g, const orc_params *p, const float *xyz, int64_t n,
                              const double *poses, int n_poses, int64_t period, int ds,
                              orc_stats *st_out)
{
    orc_stats st;
    memset(&st, 0, sizeof st);
    if (p->kernel_size < 1 || (p->kernel_size & 1) == 0 || n_poses < 1 || period < 1 || ds < 1)
        return -1;
    int64_t nv = g->nx * g->ny * g->nz;
    uint8_t *seen = NULL;
    if (p->dedup_first) {
        seen = (uint8_t *)calloc((size_t)((nv + 7) / 8), 1);
        if (!seen)
            return -1;
    }
    st.n_input = n;
    for (int64_t i = 0; i < n; i++) {
        if (i % ds != 0)
            continue;
        int64_t m = ((i % period) * (int64_t)n_poses) / period;
        int64_t c[3];
        int b, valid;
        int inside = orc_contact(p, g, xyz + 3 * i, poses + 12 * m, c, &b, &valid);
        st.n_valid += valid;
        if (!inside)
            continue;
        st.n_inside++;
        if (seen) {
            int64_t v = (c[2] * g->ny + c[1]) * g->nx + c[0];
            if (seen[v >> 3] & (1u << (v & 7)))
                continue;
            seen[v >> 3] |= (uint8_t)(1u << (v & 7));
        }
        st.n_kept++;
        orc_apply_kernel(g, p, c, b, &st);
    }
    free(seen);
    if (st_out)
        *st_out = st;
    return st.n_kept;
}

int64_t orc_integrate_scan(orc_grid *g, const orc_params *p, const float *xyz, int64_t n,
                           const double pose[12], orc_stats *st_out)
{
    return orc_integrate_scan_ex(g, p, xyz, n, pose, 1, 1, 1, st_out);
}

/* Pose at time fraction tau in [0, 1] of a sweep that starts at T0 and ends
 * at T1 (row-major 3x4 [R | t]), for the motion compensation of Sec. III-C
 * ("yaw-only or full SE(3)"; the paper gives no formula, this is a reading):
 *   mode 0, full: R(tau) = R0 Exp(tau Log(R0^T R1)) -- rotation at constant
 *     angular velocity about a fixed axis (Rodrigues' formula) -- and
 *     t(tau) = t0 + tau (t1 - t0);
 *   mode 1, yaw-only: R(tau) = Rz(tau dpsi) R0 with dpsi = yaw(R1) - yaw(R0)
 *     wrapped into (-pi, pi], yaw(R) = atan2(R_10, R_00); t(tau) as above.  */
void orc_pose_interp(const double T0[12], const double T1[12], double tau, int mode,
                     double out[12])
{
    double R0[3][3], R1[3][3], Q[3][3];
    for (int r = 0; r < 3; r++)
        for (int c = 0; c < 3; c++) {
            R0[r][c] = T0[4 * r + c];
            R1[r][c] = T1[4 * r + c];
        }
    double K[3][3] = {{0}};
    double phi = 0.0;
    if (mode == 1) {
        double dpsi = atan2(R1[1][0], R1[0][0]) - atan2(R0[1][0], R0[0][0]);
        while (dpsi > ORC_PI)
            dpsi -= 2.0 * ORC_PI;
        while (dpsi <= -ORC_PI)
            dpsi += 2.0 * ORC_PI;
        phi = tau * dpsi;
        /* Rz(phi) R0: the axis is the map's z, applied on the left */
        double cz = cos(phi), sz = sin(phi);
        for (int c = 0; c < 3; c++) {
            Q[0][c] = cz * R0[0][c] - sz * R0[1][c];
            Q[1][c] = sz * R0[0][c] + cz * R0[1][c];
            Q[2][c] = R0[2][c];
        }
    } else {
        /* D = R0^T R1, its angle and unit axis */
        double D[3][3];
        for (int r = 0; r < 3; r++)
            for (int c = 0; c < 3; c++)
                D[r][c] = R0[0][r] * R1[0][c] + R0[1][r] * R1[1][c] + R0[2][r] * R1[2][c];
        double cth = (D[0][0] + D[1][1] + D[2][2] - 1.0) / 2.0;
        if (cth > 1.0)
            cth = 1.0;
        if (cth < -1.0)
            cth = -1.0;
        double th = acos(cth);
        double w[3] = {0.0, 0.0, 0.0};
        if (th > 1e-12) {
            if (th < ORC_PI - 1e-6) {
                double k = 1.0 / (2.0 * sin(th));
                w[0] = (D[2][1] - D[1][2]) * k;
                w[1] = (D[0][2] - D[2][0]) * k;
                w[2] = (D[1][0] - D[0][1]) * k;
            } else {
                /* near a half turn: D ~ 2 w w^T - I, take the largest column */
                int j = 0;
                for (int a = 1; a < 3; a++)
                    if (D[a][a] > D[j][j])
                        j = a;
                for (int a = 0; a < 3; a++)
                    w[a] = (D[a][j] + (a == j ? 1.0 : 0.0));
                double sgn = (D[(j + 2) % 3][(j + 1) % 3] - D[(j + 1) % 3][(j + 2) % 3]) < 0.0 ? -1.0 : 1.0;
                double nw = sqrt(w[0] * w[0] + w[1] * w[1] + w[2] * w[2]);
                for (int a = 0; a < 3; a++)
                    w[a] = sgn * w[a] / nw;
            }
        }
        phi = tau * th;
        K[0][1] = -w[2];
        K[0][2] = w[1];
        K[1][0] = w[2];
        K[1][2] = -w[0];
        K[2][0] = -w[1];
        K[2][1] = w[0];
        /* Exp = I + sin(phi) K + (1 - cos(phi)) K^2, then Q = R0 Exp */
        double E[3][3];
        double s = sin(phi), c1 = 1.0 - cos(phi);
        for (int r = 0; r < 3; r++)
            for (int c = 0; c < 3; c++) {
                double kk = K[r][0] * K[0][c] + K[r][1] * K[1][c] + K[r][2] * K[2][c];
                E[r][c] = (r == c ? 1.0 : 0.0) + s * K[r][c] + c1 * kk;
            }
        for (int r = 0; r < 3; r++)
            for (int c = 0; c < 3; c++)
                Q[r][c] = R0[r][0] * E[0][c] + R0[r][1] * E[1][c] + R0[r][2] * E[2][c];
    }
    for (int r = 0; r < 3; r++) {
        for (int c = 0; c < 3; c++)
            out[4 * r + c] = Q[r][c];
        out[4 * r + 3] = T0[4 * r + 3] + tau * (T1[4 * r + 3] - T0[4 * r + 3]);
    }
}

/* ------------------------------------------------------------------ */
/* Sampled check for grids too large to integrate whole: the state of single
 * voxels after a sequence of scans, from the same definitions.  A voxel's
 * final state depends only on the kept returns whose neighbourhood covers
 * it, folded in scan order; the first-return rule only needs the contact
 * voxels seen so far in the same scan, kept here in a small hash set.
 *
 * Step 1: orc_scan_kept() lists the kept returns of one scan (contact voxel
 * and bin) in array order.
 * Step 2: orc_query_voxels() folds Eqs. 4-6 over such lists for each query
 * voxel, starting from the given state.                                 */
typedef struct {
    uint64_t *keys;
    int64_t cap;
} orc_set;

static int orc_set_insert(orc_set *s, uint64_t key)
{
    /* returns 1 when key was new; keys are stored + 1 so that 0 is empty */
    uint64_t k = key + 1;
    uint64_t h = (k * 0x9E3779B97F4A7C15ull) >> 20;
    for (int64_t probe = 0; probe < s->cap; probe++) {
        int64_t slot = (int64_t)((h + (uint64_t)probe) & (uint64_t)(s->cap - 1));
        if (s->keys[slot] == k)
            return 0;
        if (s->keys[slot] == 0) {
            s->keys[slot] = k;
            return 1;
        }
    }
    return -1;
}

/* Writes up to n kept returns: c_out[3*m..3*m+2] contact voxel, b_out[m] bin.
 * Returns the count, or -1 on failure.                                  */
int64_t orc_scan_kept(const orc_params *p, const orc_grid *g, const float *xyz, int64_t n,
                      const double pose[12], int64_t *c_out, int32_t *b_out)
{
    orc_set set = {NULL, 1};
    while (set.cap < 2 * n + 2)
        set.cap <<= 1;
    if (p->dedup_first) {
        set.keys = (uint64_t *)calloc((size_t)set.cap, sizeof(uint64_t));
        if (!set.keys)
            return -1;
    }
    int64_t m = 0;
    for (int64_t i = 0; i < n; i++) {
        int64_t c[3];
        int b, valid;
        if (!orc_contact(p, g, xyz + 3 * i, pose, c, &b, &valid))
            continue;
        if (p->dedup_first) {
            uint64_t key = (uint64_t)((c[2] * g->ny + c[1]) * g->nx + c[0]);
            int r = orc_set_insert(&set, key);
            if (r < 0) {
                free(set.keys);
                return -1;
            }
            if (r == 0)
                continue;
        }
        c_out[3 * m + 0] = c[0];
        c_out[3 * m + 1] = c[1];
        c_out[3 * m + 2] = c[2];
        b_out[m] = b;
        m++;
    }
    free(set.keys);
    return m;
}

/* Folds the kept returns (already in scan order, several scans concatenated)
 * into the state of each query voxel q[3*j..3*j+2].  mask/sign/hits hold the
 * starting state on entry and the final state on return.                */
void orc_query_voxels(const orc_params *p, int64_t n_kept, const int64_t *c, const int32_t *b,
                      int64_t nq, const int64_t *q, uint32_t *mask, uint8_t *sign, uint16_t *hits)
{
    int R = (p->kernel_size - 1) / 2;
    for (int64_t j = 0; j < nq; j++) {
        uint32_t m = mask[j];
        int h = hits[j];
        int s = sign[j];
        for (int64_t i = 0; i < n_kept; i++) {
            int64_t ox = q[3 * j + 0] - c[3 * i + 0];
            int64_t oy = q[3 * j + 1] - c[3 * i + 1];
            int64_t oz = q[3 * j + 2] - c[3 * i + 2];
            if (ox < -R || ox > R || oy < -R || oy > R || oz < -R || oz > R)
                continue;
            uint32_t k = orc_distance_mask((int)ox, (int)oy, (int)oz);
            if (m != (m & k))
                m &= k;
            if (orc_in_shadow(p, b[i], (int)ox, (int)oy, (int)oz)) {
                int h_new = h + 1;
                if (h_new > p->hit_max)
                    h_new = p->hit_max;
                if (h < p->hit_threshold && h_new >= p->hit_threshold)
                    s = 0;
                h = h_new;
            }
        }
        mask[j] = m;
        hits[j] = (uint16_t)h;
        sign[j] = (uint8_t)s;
    }
}

/* Proposed readout (the paper gives none; parity unpinned): distance in
 * voxels = popcount(mask) (Sec. III-A: the distance is the number of set
 * bits), signed by the sign flag (1 free -> +, 0 occupied -> -), times res. */
double orc_signed_distance(uint32_t mask, uint8_t sign, double res)
{
    int bits = 0;
    for (int i = 0; i < 32; i++)
        bits += (mask >> i) & 1u;
    return (sign ? 1.0 : -1.0) * (double)bits * res;
}

/* ------------------------------------------------------------------ */
/* Map export (Sec. III-C, Fig. 3): a triangle mesh of the iso-surface
 * sdf = iso by Marching Cubes, the paper's export at iso = 0.
 *
 * Readings (the paper names the method only):
 *   - the field at a voxel centre is f = (sign ? +1 : -1) * popcount(mask)
 *     * res evaluated in binary32 (res and iso rounded to float once); a
 *     cell is the cube between 2 x 2 x 2 neighbouring centres, corner q
 *     (bit 0: +x, bit 1: +y, bit 2: +z); a corner is inside when f < iso.
 *   - the vertex on a crossed edge is linearly interpolated from its lower
 *     corner a to its upper corner b: t = (iso - f_a) / (f_b - f_a),
 *     coordinate = origin + res * ((index of a + 0.5) + t) along the edge's
 *     axis, origin + res * (index + 0.5) on the other two; every operation
 *     in binary32 in this order (the mesh is a float mesh).
 *   - the configuration table is derived from the cube: on each face, every
 *     inside corner region (boundary walked counter-clockwise seen from
 *     outside) is closed by a segment from the crossing where the walk
 *     leaves it to the crossing where it entered it, so on a face with two
 *     diagonal inside corners the inside corners stay apart; the same rule on
 *     both cells sharing a face makes the surface closed.  The segments form
 *     loops, walked from the lowest-numbered edge.  A loop is cut into a fan
 *     from its first vertex whose diagonals all avoid joining two edges of
 *     one face (such a diagonal would lie in the face, where the neighbouring
 *     cell's surface meets it); with that apex first, (e_0 .. e_m-1) becomes
 *     (e_0, e_i+1, e_i), i = 1 .. m-2, whose right-hand normal points to the
 *     outside (sdf > iso).
 *   - triangles are listed by cell in x-fastest order over the box, then in
 *     table order.                                                       */

#define ORC_MC_MAXT 12

static int orc_mc_ntri[256];
static int orc_mc_tri[256][ORC_MC_MAXT][3];
static int orc_mc_built = 0;

/* the 12 edges as (lower corner, upper corner): 4 along x, 4 along y, 4 along z */
static const int orc_mc_edge_corner[12][2] = {
    {0, 1}, {2, 3}, {4, 5}, {6, 7},
    {0, 2}, {1, 3}, {4, 6}, {5, 7},
    {0, 4}, {1, 5}, {2, 6}, {3, 7}};

/* faces -x, +x, -y, +y, -z, +z; corners counter-clockwise seen from outside */
static const int orc_mc_face[6][4] = {
    {0, 4, 6, 2}, {1, 3, 7, 5}, {0, 1, 5, 4}, {2, 6, 7, 3}, {0, 2, 3, 1}, {4, 5, 7, 6}};

static int orc_mc_edge_of(int a, int b)
{
    for (int e = 0; e < 12; e++)
        if ((orc_mc_edge_corner[e][0] == a && orc_mc_edge_corner[e][1] == b) ||
            (orc_mc_edge_corner[e][0] == b && orc_mc_edge_corner[e][1] == a))
            return e;
    return -1;
}

/* 1 when edges e and f lie on a common face of the cube */
static int orc_mc_share_face(int e, int f)
{
    for (int k = 0; k < 6; k++) {
        int ne = 0, nf = 0;
        for (int c = 0; c < 4; c++) {
            int q = orc_mc_face[k][c];
            ne += q == orc_mc_edge_corner[e][0] || q == orc_mc_edge_corner[e][1];
            nf += q == orc_mc_edge_corner[f][0] || q == orc_mc_edge_corner[f][1];
        }
        if (ne == 2 && nf == 2)
            return 1;
    }
    return 0;
}

static void orc_mc_build(void)
{
    for (int cfg = 0; cfg < 256; cfg++) {
        int next[12];
        for (int e = 0; e < 12; e++)
            next[e] = -1;
        for (int f = 0; f < 6; f++) {
            int in[4], edge[4];
            for (int k = 0; k < 4; k++) {
                in[k] = (cfg >> orc_mc_face[f][k]) & 1;
                edge[k] = orc_mc_edge_of(orc_mc_face[f][k], orc_mc_face[f][(k + 1) % 4]);
            }
            /* side k runs from corner k to corner k+1: it leaves an inside
             * region when in[k] && !in[k+1], enters one when the reverse */
            for (int k = 0; k < 4; k++) {
                if (!(in[k] && !in[(k + 1) % 4]))
                    continue;
                for (int back = 1; back <= 4; back++) {
                    int j = (k - back + 4) % 4;
                    if (!in[j] && in[(j + 1) % 4]) {
                        next[edge[k]] = edge[j];
                        break;
                    }
                }
            }
        }
        int used[12] = {0};
        int nt = 0;
        for (int e0 = 0; e0 < 12; e0++) {
            if (next[e0] < 0 || used[e0])
                continue;
            int loop[12], m = 0;
            int e = e0;
            while (!used[e]) {
                used[e] = 1;
                loop[m++] = e;
                e = next[e];
            }
            int apex = 0;
            for (int a = 0; a < m; a++) {
                int ok = 1;
                for (int k = 2; k + 1 < m; k++)
                    if (orc_mc_share_face(loop[a], loop[(a + k) % m]))
                        ok = 0;
                if (ok) {
                    apex = a;
                    break;
                }
            }
            int r[12];
            for (int i = 0; i < m; i++)
                r[i] = loop[(apex + i) % m];
            for (int i = 1; i + 1 < m; i++) {
                orc_mc_tri[cfg][nt][0] = r[0];
                orc_mc_tri[cfg][nt][1] = r[i + 1];
                orc_mc_tri[cfg][nt][2] = r[i];
                nt++;
            }
        }
        orc_mc_ntri[cfg] = nt;
    }
    orc_mc_built = 1;
}

/* Triangles of configuration cfg (bit q set: corner q inside) as edge ids;
 * returns their number.  tri may be NULL.                                 */
int orc_mc_config(int cfg, int *tri)
{
    if (!orc_mc_built)
        orc_mc_build();
    if (tri)
        for (int t = 0; t < orc_mc_ntri[cfg]; t++)
            for (int v = 0; v < 3; v++)
                tri[3 * t + v] = orc_mc_tri[cfg][t][v];
    return orc_mc_ntri[cfg];
}

static double orc_sdf_at(const orc_grid *g, int64_t x, int64_t y, int64_t z)
{
    int64_t v = (z * g->ny + y) * g->nx + x;
    return orc_signed_distance(g->mask[v], g->sign[v], g->res);
}

/* the mesh's binary32 field value of a voxel */
static float orc_mesh_level(const orc_grid *g, int64_t x, int64_t y, int64_t z, float res)
{
    int64_t v = (z * g->ny + y) * g->nx + x;
    int bits = 0;
    for (int i = 0; i < 32; i++)
        bits += (g->mask[v] >> i) & 1u;
    return (g->sign[v] ? 1.0f : -1.0f) * (float)bits * res;
}

/* Signed distance of every voxel of the box [x0, x0+bx) x [y0, y0+by) x
 * [z0, z0+bz) into out[(z * by + y) * bx + x] (float).                    */
void orc_sdf_field(const orc_grid *g, const int64_t box[6], float *out)
{
    for (int64_t z = 0; z < box[5]; z++)
        for (int64_t y = 0; y < box[4]; y++)
            for (int64_t x = 0; x < box[3]; x++)
                out[(z * box[4] + y) * box[3] + x] =
                    (float)orc_sdf_at(g, box[0] + x, box[1] + y, box[2] + z);
}

/* Marching Cubes over the cells of the voxel box (x0, y0, z0, bx, by, bz):
 * cells (i, j, k) with corners inside the box, numbered
 * L = (k (by - 1) + j) (bx - 1) + i.  Writes up to max_tri triangles (9
 * floats each: three xyz vertices in the map frame) to tri and, if cell is
 * not NULL, the cell number L of each; returns the total number of
 * triangles of the box.                                                   */
int64_t orc_mesh(const orc_grid *g, const int64_t box[6], double iso, float *tri,
                 int64_t max_tri, int64_t *cell)
{
    if (!orc_mc_built)
        orc_mc_build();
    int64_t cx = box[3] - 1, cy = box[4] - 1, cz = box[5] - 1;
    if (cx < 1 || cy < 1 || cz < 1)
        return 0;
    float res = (float)g->res, isof = (float)iso;
    float org[3] = {(float)g->origin[0], (float)g->origin[1], (float)g->origin[2]};
    int64_t n = 0;
    for (int64_t k = 0; k < cz; k++)
        for (int64_t j = 0; j < cy; j++)
            for (int64_t i = 0; i < cx; i++) {
                int64_t base[3] = {box[0] + i, box[1] + j, box[2] + k};
                float f[8];
                int cfg = 0;
                for (int q = 0; q < 8; q++) {
                    f[q] = orc_mesh_level(g, base[0] + (q & 1), base[1] + ((q >> 1) & 1),
                                          base[2] + ((q >> 2) & 1), res);
                    if (f[q] < isof)
                        cfg |= 1 << q;
                }
                for (int t = 0; t < orc_mc_ntri[cfg]; t++, n++) {
                    if (n >= max_tri)
                        continue;
                    for (int v = 0; v < 3; v++) {
                        int e = orc_mc_tri[cfg][t][v];
                        int a = orc_mc_edge_corner[e][0], b = orc_mc_edge_corner[e][1];
                        int axis = e / 4;
                        float tt = (isof - f[a]) / (f[b] - f[a]);
                        for (int d = 0; d < 3; d++) {
                            float idx = (float)(base[d] + ((a >> d) & 1)) + 0.5f;
                            if (d == axis)
                                idx = idx + tt;
                            tri[9 * n + 3 * v + d] = org[d] + res * idx;
                        }
                    }
                    if (cell)
                        cell[n] = (k * cy + j) * cx + i;
                }
            }
    return n;
}

/* ------------------------------------------------------------------ */
/* Reconstruction quality (Sec. IV-B, "Mapping results"): nearest-neighbour
 * distances between a predicted point set (sampled from the iso-surface of
 * the reconstructed mesh) and the reference surface points.
 *   accuracy     = mean over predicted points of the distance to the
 *                  nearest reference point;
 *   completeness = mean over reference points of the distance to the
 *                  nearest predicted point;
 *   Chamfer-L1   = (accuracy + completeness) / 2;
 *   recall       = fraction of reference points within the tolerance t of
 *                  the prediction, precision the same for predicted points
 *                  against the reference, F-score their harmonic mean.
 * Reading: "within the tolerance" is d < t; F = 0 when P + R = 0.        */

/* out[i] = min over reference points of |query_i - ref_j| (binary64,
 * brute force; +inf when there is no reference point)                     */
void orc_nn_distances(const float *ref, int64_t n_ref, const float *q, int64_t n_q, double *out)
{
    for (int64_t i = 0; i < n_q; i++) {
        double best = INFINITY;
        for (int64_t j = 0; j < n_ref; j++) {
            double dx = (double)q[3 * i] - (double)ref[3 * j];
            double dy = (double)q[3 * i + 1] - (double)ref[3 * j + 1];
            double dz = (double)q[3 * i + 2] - (double)ref[3 * j + 2];
            double d2 = dx * dx + dy * dy + dz * dz;
            if (d2 < best)
                best = d2;
        }
        out[i] = sqrt(best);
    }
}

/* out: accuracy, completeness, Chamfer-L1, precision, recall, F-score,
 * from the two distance lists of orc_nn_distances.                        */
void orc_quality_from_distances(const double *d_pred, int64_t n_pred, const double *d_gt,
                                int64_t n_gt, double t, double out[6])
{
    double sa = 0.0, sc = 0.0;
    int64_t np_in = 0, ng_in = 0;
    for (int64_t i = 0; i < n_pred; i++) {
        sa += d_pred[i];
        np_in += d_pred[i] < t;
    }
    for (int64_t i = 0; i < n_gt; i++) {
        sc += d_gt[i];
        ng_in += d_gt[i] < t;
    }
    double acc = n_pred ? sa / (double)n_pred : 0.0;
    double comp = n_gt ? sc / (double)n_gt : 0.0;
    double prec = n_pred ? (double)np_in / (double)n_pred : 0.0;
    double rec = n_gt ? (double)ng_in / (double)n_gt : 0.0;
    out[0] = acc;
    out[1] = comp;
    out[2] = (acc + comp) / 2.0;
    out[3] = prec;
    out[4] = rec;
    out[5] = prec + rec > 0.0 ? 2.0 * prec * rec / (prec + rec) : 0.0;
}
