// C ABI entry points (include/dbtsdf.h): argument checks, the host build of
// the directional kernel tables, workspace layout, and the launch sequence
// of one scan.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "dbt_internal.cuh"

using namespace dbt;

// pi rounded to the nearest binary64 value
static const double kPi = 3.14159265358979323846;

// ------------------------------------------------------------------ errors
// A fixed per-thread buffer: reporting an error never allocates.
static thread_local char t_err[512];

static dbt_status fail(dbt_status st, const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(t_err, sizeof t_err, fmt, ap);
    va_end(ap);
    return st;
}

static dbt_status cuda_fail(cudaError_t e, const char *what) {
    return fail(DBT_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

dbt_status dbt::report_cuda_error(cudaError_t e, const char *what) { return cuda_fail(e, what); }

#define DBT_CUDA(call)                                   \
    do {                                                 \
        cudaError_t e_ = (call);                         \
        if (e_ != cudaSuccess) return cuda_fail(e_, #call); \
    } while (0)

static bool aligned256(const void *p) { return ((uintptr_t)p & 255u) == 0; }

// ------------------------------------------------------------------ tables
static int ceil_isqrt(int n);

struct dbt_kernels {
    dbt_params params;
    DevParams dp;
    DevTables dt;
    void *d_base = nullptr;
    std::vector<uint32_t> m2;         // mask by r^2
    std::vector<uint32_t> sh_off;     // packed shadow offsets by bin
    std::vector<uint32_t> sh_start;   // nbins + 1
    std::vector<uint32_t> prow;       // kernel-row codes for the integration kernel
};

// Kernel-row codes: for q = oy^2 + oz^2 in [0, 2 R^2] and s in [0, 2R + 4),
// the four bytes of P[q][s] are the Eq. 3 distance codes ceil(sqrt(ox^2 + q))
// of the voxels at ox = s - 3 - R + e (e = 0..3), and 32 (no change) where
// |ox| > R.  A 4-voxel word whose first voxel is at kernel offset ox reads
// P[q][ox + R + 3].
static void build_row_codes(int R, std::vector<uint32_t> &prow) {
    const int W = 2 * R + 4;
    prow.assign((size_t)(2 * R * R + 1) * W, 0u);
    for (int q = 0; q <= 2 * R * R; ++q)
        for (int s = 0; s < W; ++s) {
            uint32_t word = 0;
            for (int e = 0; e < 4; ++e) {
                const int t = s - 3 + e;
                uint32_t k = 32u;
                if (t >= 0 && t <= 2 * R) {
                    const int ox = t - R;
                    k = (uint32_t)ceil_isqrt(ox * ox + q);
                }
                word |= k << (8 * e);
            }
            prow[(size_t)q * W + s] = word;
        }
}

// Smallest k with k * k >= n (exact integer ceil of sqrt).
static int ceil_isqrt(int n) {
    int k = 0;
    while (k * k < n) ++k;
    return k;
}

// Eq. 3 as a function of r^2 = |o|^2: 0 at the centre, else ceil(r) low bits.
static uint32_t eq3_mask_of_r2(int r2) {
    int k = ceil_isqrt(r2);
    if (k == 0) return 0u;
    if (k >= 32) return 0xFFFFFFFFu;
    return 0xFFFFFFFFu >> (32 - k);
}

// Octahedral cell centre decoded to a direction, times n (integer vector).
static void octa_dir_int(int b, int n, long long v[3]) {
    long long U = 2 * (b % n) + 1 - n;
    long long V = 2 * (b / n) + 1 - n;
    long long Z = n - std::llabs(U) - std::llabs(V);
    if (Z < 0) {
        long long fu = (n - std::llabs(V)) * (U < 0 ? -1 : 1);
        long long fv = (n - std::llabs(U)) * (V < 0 ? -1 : 1);
        U = fu;
        V = fv;
    }
    v[0] = U;
    v[1] = V;
    v[2] = Z;
}

static double az_edge(int k, int baz) { return ((2.0 * kPi) * (double)k) / (double)baz; }
static double el_edge(int k, int bel) { return (kPi * (double)k) / (double)bel - kPi / 2.0; }

static dbt_status check_params(const dbt_params *p) {
    if (!p) return fail(DBT_EINVAL, "params is NULL");
    if (p->kernel_size < 1 || p->kernel_size > MAX_K || (p->kernel_size & 1) == 0)
        return fail(DBT_EINVAL, "kernel_size must be odd in [1, %d], got %d", MAX_K, p->kernel_size);
    if (p->scheme == DBT_BINS_OCTA) {
        if (p->bins_a < 1 || p->bins_a > 64 || p->bins_b != p->bins_a)
            return fail(DBT_EINVAL, "octahedral bins need bins_a == bins_b in [1, 64]");
    } else if (p->scheme == DBT_BINS_AZEL) {
        if (p->bins_a < 1 || p->bins_a > MAX_EDGES || p->bins_b < 1 || p->bins_b > MAX_EDGES)
            return fail(DBT_EINVAL, "az/el bins must be in [1, %d]", MAX_EDGES);
    } else {
        return fail(DBT_EINVAL, "unknown bin scheme %d", p->scheme);
    }
    if (!(p->shadow_radius >= 0.0) || !std::isfinite(p->shadow_radius))
        return fail(DBT_EINVAL, "shadow_radius must be finite and >= 0");
    if (p->hit_max < 1 || p->hit_max > 65535)
        return fail(DBT_EINVAL, "hit_max must be in [1, 65535]");
    if (p->hit_threshold < 1 || p->hit_threshold > p->hit_max)
        return fail(DBT_EINVAL, "hit_threshold must be in [1, hit_max]");
    if (p->dedup_first != 0 && p->dedup_first != 1)
        return fail(DBT_EINVAL, "dedup_first must be 0 or 1");
    if (p->reserved != 0) return fail(DBT_EINVAL, "reserved must be 0");
    if (!(p->shadow_cos >= 0.0 && p->shadow_cos <= 1.0))
        return fail(DBT_EINVAL, "shadow_cos must be in [0, 1]");
    return DBT_OK;
}

// Shadow membership of offset o for bin b (Sec. III-B): |o|^2 <= r_s^2 and
// o . v_b >= c sqrt(|o|^2 |v_b|^2), c = shadow_cos (0: the hemisphere).
// Octahedral v_b is the integer decode of the cell centre (n times u_b), so
// the hemisphere's sign test is exact; the cone compares in binary64.
static bool in_shadow(const dbt_params *p, const double azel_u[3], const long long octa_v[3],
                      int ox, int oy, int oz) {
    double r2 = (double)ox * ox + (double)oy * oy + (double)oz * oz;
    if (!(r2 <= p->shadow_radius * p->shadow_radius)) return false;
    double v[3];
    for (int i = 0; i < 3; ++i)
        v[i] = p->scheme == DBT_BINS_OCTA ? (double)octa_v[i] : azel_u[i];
    const double dot = ((double)ox * v[0] + (double)oy * v[1]) + (double)oz * v[2];
    if (p->shadow_cos == 0.0) return dot >= 0.0;
    const double vv = (v[0] * v[0] + v[1] * v[1]) + v[2] * v[2];
    return dot >= p->shadow_cos * std::sqrt(r2 * vv);
}

// Host tables: Eq. 3 masks by r^2 and the per-bin shadow offset lists.
static void build_host_tables(const dbt_params *p, std::vector<uint32_t> &m2,
                              std::vector<uint32_t> &sh_off, std::vector<uint32_t> &sh_start) {
    const int K = p->kernel_size, R = (K - 1) / 2;
    const int nbins = p->bins_a * p->bins_b;
    m2.assign(3 * R * R + 1, 0u);
    for (int r2 = 0; r2 <= 3 * R * R; ++r2) m2[r2] = eq3_mask_of_r2(r2);
    sh_off.clear();
    sh_start.assign(nbins + 1, 0u);
    for (int b = 0; b < nbins; ++b) {
        sh_start[b] = (uint32_t)sh_off.size();
        double u[3] = {0, 0, 0};
        long long v[3] = {0, 0, 0};
        if (p->scheme == DBT_BINS_OCTA) {
            octa_dir_int(b, p->bins_a, v);
        } else {
            const int a = b % p->bins_a, e = b / p->bins_a;
            const double alpha = ((2.0 * kPi) * ((double)a + 0.5)) / (double)p->bins_a;
            const double eps = (kPi * ((double)e + 0.5)) / (double)p->bins_b - kPi / 2.0;
            u[0] = std::cos(eps) * std::cos(alpha);
            u[1] = std::cos(eps) * std::sin(alpha);
            u[2] = std::sin(eps);
        }
        for (int oz = -R; oz <= R; ++oz)
            for (int oy = -R; oy <= R; ++oy)
                for (int ox = -R; ox <= R; ++ox)
                    if (in_shadow(p, u, v, ox, oy, oz)) sh_off.push_back(pack_off(ox, oy, oz));
    }
    sh_start[nbins] = (uint32_t)sh_off.size();
}

// Dense export of host tables: K^3 masks and bins x K^3 shadow bytes.
static void export_tables(int K, int nbins, const std::vector<uint32_t> &m2,
                          const std::vector<uint32_t> &sh_off, const std::vector<uint32_t> &sh_start,
                          uint32_t *h_mask, uint8_t *h_shadow) {
    const int R = (K - 1) / 2;
    if (h_mask) {
        for (int oz = -R; oz <= R; ++oz)
            for (int oy = -R; oy <= R; ++oy)
                for (int ox = -R; ox <= R; ++ox)
                    h_mask[((oz + R) * K + (oy + R)) * K + (ox + R)] = m2[ox * ox + oy * oy + oz * oz];
    }
    if (h_shadow) {
        const size_t kk = (size_t)K * K * K;
        memset(h_shadow, 0, kk * nbins);
        for (int b = 0; b < nbins; ++b)
            for (uint32_t e = sh_start[b]; e < sh_start[b + 1]; ++e) {
                const uint32_t o = sh_off[e];
                const int ox = off_axis(o, 0), oy = off_axis(o, 1), oz = off_axis(o, 2);
                h_shadow[b * kk + ((oz + R) * K + (oy + R)) * K + (ox + R)] = 1;
            }
    }
}

extern "C" dbt_status dbt_tables_host(const dbt_params *p, uint32_t *h_mask, uint8_t *h_shadow) {
    dbt_status st = check_params(p);
    if (st != DBT_OK) return st;
    std::vector<uint32_t> m2, sh_off, sh_start;
    build_host_tables(p, m2, sh_off, sh_start);
    export_tables(p->kernel_size, p->bins_a * p->bins_b, m2, sh_off, sh_start, h_mask, h_shadow);
    return DBT_OK;
}

extern "C" dbt_status dbt_kernels_build(const dbt_params *p, dbt_kernels **out) {
    if (!out) return fail(DBT_EINVAL, "out is NULL");
    *out = nullptr;
    dbt_status st = check_params(p);
    if (st != DBT_OK) return st;
    dbt_kernels *k = new (std::nothrow) dbt_kernels();
    if (!k) return fail(DBT_ENOMEM, "host allocation failed");
    k->params = *p;
    const int K = p->kernel_size, R = (K - 1) / 2;
    const int nbins = p->bins_a * p->bins_b;
    build_host_tables(p, k->m2, k->sh_off, k->sh_start);
    build_row_codes(R, k->prow);
    // Eq. 2 edge tables
    std::vector<double> az_c(MAX_EDGES, 0.0), az_s(MAX_EDGES, 0.0), el_s(MAX_EDGES, 0.0);
    std::vector<int> az_up(MAX_EDGES, 0);
    if (p->scheme == DBT_BINS_AZEL) {
        for (int j = 1; j < p->bins_a; ++j) {
            const double th = az_edge(j, p->bins_a);
            az_c[j] = std::cos(th);
            az_s[j] = std::sin(th);
            az_up[j] = th < kPi;
        }
        for (int j = 1; j < p->bins_b; ++j) el_s[j] = std::sin(el_edge(j, p->bins_b));
    }
    // Shadow sub-ranges.  Each bin's offsets are listed oz-major (sh_off, as
    // built) and again oy-major (sh_y); sh_zs[b * (sw + 1) + k] is the first
    // entry of bin b's oz-major list with oz >= k - sr (k = 0 .. sw), sh_ys
    // the same for oy in the oy-major list.  A pair whose contact lies
    // outside its brick along z (or y) then walks only the entries whose
    // plane (or row) falls in the brick.
    const int sr = std::min(R, (int)std::floor(p->shadow_radius));
    const int sw = 2 * sr + 1;
    std::vector<uint32_t> sh_y(k->sh_off.size()), sh_zs((size_t)nbins * (sw + 1)),
        sh_ys((size_t)nbins * (sw + 1));
    for (int b = 0; b < nbins; ++b) {
        const uint32_t e0 = k->sh_start[b], e1 = k->sh_start[b + 1];
        std::vector<uint32_t> by(k->sh_off.begin() + e0, k->sh_off.begin() + e1);
        std::stable_sort(by.begin(), by.end(), [](uint32_t a, uint32_t c) {
            return off_axis(a, 1) != off_axis(c, 1) ? off_axis(a, 1) < off_axis(c, 1)
                                                    : off_axis(a, 2) < off_axis(c, 2);
        });
        std::copy(by.begin(), by.end(), sh_y.begin() + e0);
        for (int kk = 0; kk <= sw; ++kk) {
            uint32_t ez = e0, ey = e0;
            while (ez < e1 && off_axis(k->sh_off[ez], 2) < kk - sr) ++ez;
            while (ey < e1 && off_axis(sh_y[ey], 1) < kk - sr) ++ey;
            sh_zs[(size_t)b * (sw + 1) + kk] = ez;
            sh_ys[(size_t)b * (sw + 1) + kk] = ey;
        }
    }
    // one device block for all tables
    const size_t n_m2 = k->m2.size(), n_off = std::max<size_t>(1, k->sh_off.size());
    size_t off_m2 = 0;
    size_t off_sh = off_m2 + ((n_m2 * 4 + 255) & ~size_t(255));
    size_t off_st = off_sh + ((n_off * 4 + 255) & ~size_t(255));
    size_t off_azc = off_st + (((nbins + 1) * 4 + 255) & ~size_t(255));
    size_t off_azs = off_azc + MAX_EDGES * 8;
    size_t off_els = off_azs + MAX_EDGES * 8;
    size_t off_up = off_els + MAX_EDGES * 8;
    size_t off_pr = off_up + MAX_EDGES * 4;
    size_t off_shy = off_pr + ((k->prow.size() * 4 + 255) & ~size_t(255));
    size_t off_zs = off_shy + ((n_off * 4 + 255) & ~size_t(255));
    size_t off_ys = off_zs + ((sh_zs.size() * 4 + 255) & ~size_t(255));
    size_t total = off_ys + sh_ys.size() * 4;
    cudaError_t e = cudaMalloc(&k->d_base, total);
    if (e != cudaSuccess) {
        delete k;
        return cuda_fail(e, "cudaMalloc(kernel tables)");
    }
    char *base = (char *)k->d_base;
    e = cudaMemcpy(base + off_m2, k->m2.data(), n_m2 * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess && !k->sh_off.empty())
        e = cudaMemcpy(base + off_sh, k->sh_off.data(), k->sh_off.size() * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(base + off_st, k->sh_start.data(), (nbins + 1) * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(base + off_azc, az_c.data(), MAX_EDGES * 8, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(base + off_azs, az_s.data(), MAX_EDGES * 8, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(base + off_els, el_s.data(), MAX_EDGES * 8, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(base + off_up, az_up.data(), MAX_EDGES * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(base + off_pr, k->prow.data(), k->prow.size() * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess && !sh_y.empty())
        e = cudaMemcpy(base + off_shy, sh_y.data(), sh_y.size() * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(base + off_zs, sh_zs.data(), sh_zs.size() * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(base + off_ys, sh_ys.data(), sh_ys.size() * 4, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        cudaFree(k->d_base);
        delete k;
        return cuda_fail(e, "cudaMemcpy(kernel tables)");
    }
    k->dp.K = K;
    k->dp.R = R;
    k->dp.scheme = p->scheme;
    k->dp.na = p->bins_a;
    k->dp.nb = p->bins_b;
    k->dp.nbins = nbins;
    k->dp.T = p->hit_threshold;
    k->dp.Hmax = p->hit_max;
    k->dp.dedup = p->dedup_first;
    k->dp.n_m2 = (int)n_m2;
    k->dp.sr = sr;
    k->dp.n_sh = (int)k->sh_off.size();
    k->dt.m2 = (const uint32_t *)(base + off_m2);
    k->dt.sh_off = (const uint32_t *)(base + off_sh);
    k->dt.sh_start = (const uint32_t *)(base + off_st);
    k->dt.az_c = (const double *)(base + off_azc);
    k->dt.az_s = (const double *)(base + off_azs);
    k->dt.el_s = (const double *)(base + off_els);
    k->dt.az_up = (const int *)(base + off_up);
    k->dt.prow = (const uint32_t *)(base + off_pr);
    k->dt.sh_y = (const uint32_t *)(base + off_shy);
    k->dt.sh_zs = (const uint32_t *)(base + off_zs);
    k->dt.sh_ys = (const uint32_t *)(base + off_ys);
    *out = k;
    return DBT_OK;
}

extern "C" dbt_status dbt_kernels_destroy(dbt_kernels *k) {
    if (!k) return DBT_OK;
    cudaError_t e = k->d_base ? cudaFree(k->d_base) : cudaSuccess;
    delete k;
    if (e != cudaSuccess) return cuda_fail(e, "cudaFree(kernel tables)");
    return DBT_OK;
}

extern "C" dbt_status dbt_kernels_export(const dbt_kernels *k, uint32_t *h_mask, uint8_t *h_shadow) {
    if (!k) return fail(DBT_EINVAL, "kernels is NULL");
    export_tables(k->dp.K, k->dp.nbins, k->m2, k->sh_off, k->sh_start, h_mask, h_shadow);
    return DBT_OK;
}

// ------------------------------------------------------------------ grid
static dbt_status check_grid(const dbt_grid *g) {
    if (!g) return fail(DBT_EINVAL, "grid is NULL");
    if (!g->mask || !g->sign || !g->hits) return fail(DBT_EINVAL, "grid arrays must be non-NULL");
    if (!aligned256(g->mask) || !aligned256(g->sign) || !aligned256(g->hits))
        return fail(DBT_EINVAL, "grid arrays must be 256-byte aligned");
    if (g->nx < 1 || g->ny < 1 || g->nz < 1) return fail(DBT_EINVAL, "grid dims must be >= 1");
    if (g->pitch_x < g->nx || (g->pitch_x % 32) != 0)
        return fail(DBT_EINVAL, "pitch_x must be >= nx and a multiple of 32");
    const double nv = (double)g->pitch_x * g->ny * g->nz;
    if (nv > 1099511627776.0) return fail(DBT_EINVAL, "grid larger than 2^40 voxels");
    if (!(g->res > 0.0) || !std::isfinite(g->res)) return fail(DBT_EINVAL, "res must be > 0");
    for (int a = 0; a < 3; ++a)
        if (!std::isfinite(g->origin[a])) return fail(DBT_EINVAL, "origin must be finite");
    return DBT_OK;
}

// Grid view for bricks of depth bz (4, 8 or 16).
static DevGrid dev_grid(const dbt_grid *g, int bz = BZ_DEFAULT) {
    DevGrid d;
    d.mask = g->mask;
    d.sign = g->sign;
    d.hits = g->hits;
    d.nx = g->nx;
    d.ny = g->ny;
    d.nz = g->nz;
    d.pitch = g->pitch_x;
    d.nbx = g->pitch_x / BX;
    d.nby = (g->ny + BY - 1) / BY;
    d.nbz = (g->nz + bz - 1) / bz;
    d.bzs = bz_shift(bz);
    d.res = g->res;
    d.inv_res = 1.0 / g->res;
    d.ox = g->origin[0];
    d.oy = g->origin[1];
    d.oz = g->origin[2];
    return d;
}

extern "C" dbt_status dbt_grid_layout(int32_t nx, int32_t ny, int32_t nz, int32_t *pitch_x,
                                      size_t *mask_bytes, size_t *sign_bytes, size_t *hits_bytes) {
    if (nx < 1 || ny < 1 || nz < 1) return fail(DBT_EINVAL, "grid dims must be >= 1");
    if (nx > 0x7FFFFFE0) return fail(DBT_EINVAL, "nx too large");
    const long long pitch = ((long long)nx + 31) / 32 * 32;
    const double nv = (double)pitch * ny * nz;
    if (nv > 1099511627776.0) return fail(DBT_EINVAL, "grid larger than 2^40 voxels");
    const size_t n = (size_t)pitch * (size_t)ny * (size_t)nz;
    if (pitch_x) *pitch_x = (int32_t)pitch;
    if (mask_bytes) *mask_bytes = n * 4;
    if (sign_bytes) *sign_bytes = n;
    if (hits_bytes) *hits_bytes = n * 2;
    return DBT_OK;
}

extern "C" dbt_status dbt_grid_init(const dbt_grid *g, void *stream) {
    dbt_status st = check_grid(g);
    if (st != DBT_OK) return st;
    const size_t n = (size_t)g->pitch_x * g->ny * g->nz;
    cudaStream_t s = (cudaStream_t)stream;
    DBT_CUDA(cudaMemsetAsync(g->mask, 0xFF, n * 4, s));   // all mask bits set
    DBT_CUDA(cudaMemsetAsync(g->sign, 0x01, n, s));       // free
    DBT_CUDA(cudaMemsetAsync(g->hits, 0x00, n * 2, s));   // no hits
    return DBT_OK;
}

// ------------------------------------------------------------------ workspace
// Offsets of the scratch regions; a layout function must set every one
// (ws_bind refuses a layout with a region left unset).
constexpr size_t kUnset = ~size_t(0);
struct WsLayout {
    size_t hdr = kUnset, stage = kUnset, stage_b = kUnset, prec = kUnset, hkey = kUnset, hidx = kUnset,
           bcnt = kUnset, boff = kUnset, order = kUnset, lq0 = kUnset, lq1 = kUnset, lq2 = kUnset,
           pairs = kUnset, poses = kUnset, total = kUnset;
    uint32_t hcap_alloc = 0, max_touched = 0, nbricks = 0;
    unsigned long long pairs_cap = 0;
    bool complete() const {
        for (size_t v : {hdr, stage, stage_b, prec, hkey, hidx, bcnt, boff, order, lq0, lq1, lq2, pairs,
                         poses, total})
            if (v == kUnset || (v != total && v >= total)) return false;
        return true;
    }
};

static size_t up256(size_t v) { return (v + 255) & ~size_t(255); }


// Bricks of depth bz over a grid of pitch_x x ny x nz voxels.
static unsigned long long bricks_of(int pitch_x, int ny, int nz, int bz) {
    return (unsigned long long)(pitch_x / BX) * ((ny + BY - 1) / BY) * ((nz + bz - 1) / bz);
}

// staging: two host-input staging buffers (dbt_integrate_scan_host copies
// the next scan into one while the previous scan reads the other); the
// no-allocation entry point takes device input only and needs none.
// Scratch layout for grids of pitch_x x ny x nz voxels and kernel size K,
// with room for the brick counters and pair slots of bricks of depth bz
// (the shallowest depth a workspace may be tuned to has the most of both).
static dbt_status ws_layout_dims(int pitch_x, int ny, int nz, int K, long long max_points,
                                 WsLayout *L, bool staging, int bz) {
    if (max_points < 1 || max_points > (1ll << 30))
        return fail(DBT_EINVAL, "max_points must be in [1, 2^30]");
    const unsigned long long nb = bricks_of(pitch_x, ny, nz, bz);
    if (nb >= (1ull << 32)) return fail(DBT_EINVAL, "too many bricks");
    L->nbricks = (uint32_t)nb;
    uint32_t hc = 64;
    while (hc < 2ull * (unsigned long long)max_points) hc <<= 1;
    L->hcap_alloc = hc;
    L->pairs_cap = (unsigned long long)max_points * max_pairs_per_return(K, bz);
    L->max_touched = (uint32_t)std::min<unsigned long long>(nb, L->pairs_cap);
    size_t o = 0;
    L->hdr = o;      o += up256(sizeof(WsHeader));
    L->stage = o;    o += up256(staging ? (size_t)max_points * 12 : 16);
    L->stage_b = o;  o += up256(staging ? (size_t)max_points * 12 : 16);
    L->prec = o;     o += up256((size_t)max_points * 16);
    L->hkey = o;     o += up256((size_t)hc * 8);
    L->hidx = o;     o += up256((size_t)hc * 4);
    L->bcnt = o;     o += up256((size_t)nb * 4);
    L->boff = o;     o += up256((size_t)nb * 4);
    L->order = o;    o += up256((size_t)L->max_touched * 4);
    L->lq0 = o;      o += up256((size_t)L->max_touched * 4);
    L->lq1 = o;      o += up256((size_t)L->max_touched * 4);
    L->lq2 = o;      o += up256((size_t)L->max_touched * 4);
    L->pairs = o;    o += up256((size_t)L->pairs_cap * 4);
    L->poses = o;    o += up256((size_t)MAX_SCAN_POSES * sizeof(Pose));
    L->total = o;
    return DBT_OK;
}

static dbt_status ws_layout(const dbt_grid *g, const dbt_kernels *k, long long max_points, WsLayout *L,
                            bool staging = true, int bz = BZ_MIN) {
    return ws_layout_dims(g->pitch_x, g->ny, g->nz, k->dp.K, max_points, L, staging, bz);
}

struct dbt_workspace {
    WsLayout L;
    WsDev d;
    void *buf;
    long long max_points;
    int nx, ny, nz, pitch, K;
    cudaEvent_t ev_begin = nullptr, ev_end = nullptr;   // optional timing of the integrate kernel
    int ctas = 0;                                       // integrate grid; 0 = occupancy maximum
    int bz = BZ_DEFAULT;                                // brick depth
    // dbt_integrate_scan_host: the second staging buffer, the copy stream and
    // per buffer an event after its copy and one after the scan that read it
    float *stage_b = nullptr;
    cudaStream_t copy_stream = nullptr;
    cudaEvent_t ev_copied[2] = {nullptr, nullptr}, ev_free[2] = {nullptr, nullptr};
    int stage_next = 0;
    ~dbt_workspace() {
        for (int i = 0; i < 2; ++i) {
            if (ev_copied[i]) cudaEventDestroy(ev_copied[i]);
            if (ev_free[i]) cudaEventDestroy(ev_free[i]);
        }
        if (copy_stream) cudaStreamDestroy(copy_stream);
    }
};

extern "C" dbt_status dbt_workspace_size(const dbt_grid *g, const dbt_kernels *k, int64_t max_points,
                                         size_t *bytes) {
    if (!k) return fail(DBT_EINVAL, "kernels is NULL");
    if (!bytes) return fail(DBT_EINVAL, "bytes is NULL");
    if (!g) return fail(DBT_EINVAL, "grid is NULL");
    // only the geometry of g matters here; its arrays may still be NULL
    dbt_grid gg = *g;
    static uint32_t dummy[64] __attribute__((aligned(256)));
    if (!gg.mask) gg.mask = dummy;
    if (!gg.sign) gg.sign = (uint8_t *)dummy;
    if (!gg.hits) gg.hits = (uint16_t *)dummy;
    dbt_status st = check_grid(&gg);
    if (st != DBT_OK) return st;
    WsLayout L;
    st = ws_layout(&gg, k, max_points, &L);
    if (st != DBT_OK) return st;
    *bytes = L.total;
    return DBT_OK;
}

// Points a workspace view at the regions of base laid out by L.
static dbt_status ws_bind(dbt_workspace *w, const dbt_grid *g, const dbt_kernels *k,
                          long long max_points, const WsLayout &L, void *base_ptr) {
    if (!L.complete()) return fail(DBT_ESTATE, "internal error: incomplete scratch layout");
    char *base = (char *)base_ptr;
    w->L = L;
    w->buf = base_ptr;
    w->max_points = max_points;
    w->nx = g->nx;
    w->ny = g->ny;
    w->nz = g->nz;
    w->pitch = g->pitch_x;
    w->K = k->dp.K;
    w->d.hdr = (WsHeader *)(base + L.hdr);
    w->d.stage = (float *)(base + L.stage);
    // host staging only where the layout gave both buffers room for max_points
    w->stage_b = L.prec - L.stage_b >= (size_t)max_points * 12 ? (float *)(base + L.stage_b) : nullptr;
    w->d.prec = (int4 *)(base + L.prec);
    w->d.hkey = (unsigned long long *)(base + L.hkey);
    w->d.hidx = (uint32_t *)(base + L.hidx);
    w->d.hcap_alloc = L.hcap_alloc;
    w->d.bcnt = (uint32_t *)(base + L.bcnt);
    w->d.boff = (uint32_t *)(base + L.boff);
    w->d.order = (uint32_t *)(base + L.order);
    w->d.lq[0] = (uint32_t *)(base + L.lq0);
    w->d.lq[1] = (uint32_t *)(base + L.lq1);
    w->d.lq[2] = (uint32_t *)(base + L.lq2);
    w->d.max_touched = L.max_touched;
    w->d.pairs = (uint32_t *)(base + L.pairs);
    w->d.pairs_cap = L.pairs_cap;
    w->d.poses = (Pose *)(base + L.poses);
    w->d.heavy = HEAVY_PAIRS;
    w->bz = BZ_DEFAULT;
    w->d.nbricks = (uint32_t)bricks_of(g->pitch_x, g->ny, g->nz, BZ_DEFAULT);   // <= L.nbricks
    return DBT_OK;
}

extern "C" dbt_status dbt_workspace_create(const dbt_grid *g, const dbt_kernels *k, int64_t max_points,
                                           void *d_buf, size_t bytes, void *stream,
                                           dbt_workspace **out) {
    if (!out) return fail(DBT_EINVAL, "out is NULL");
    *out = nullptr;
    if (!k) return fail(DBT_EINVAL, "kernels is NULL");
    dbt_status st = check_grid(g);
    if (st != DBT_OK) return st;
    if (!d_buf || !aligned256(d_buf)) return fail(DBT_EINVAL, "workspace buffer must be 256-byte aligned");
    WsLayout L;
    st = ws_layout(g, k, max_points, &L);
    if (st != DBT_OK) return st;
    if (bytes < L.total)
        return fail(DBT_ENOMEM, "workspace too small: %zu < %zu bytes", bytes, L.total);
    dbt_workspace *w = new (std::nothrow) dbt_workspace();
    if (!w) return fail(DBT_ENOMEM, "host allocation failed");
    st = ws_bind(w, g, k, max_points, L, d_buf);
    if (st != DBT_OK) {
        delete w;
        return st;
    }
    cudaError_t e = cudaMemsetAsync(d_buf, 0, L.total, (cudaStream_t)stream);
    if (e != cudaSuccess) {
        delete w;
        return cuda_fail(e, "cudaMemsetAsync(workspace)");
    }
    *out = w;
    return DBT_OK;
}

extern "C" dbt_status dbt_workspace_reset(dbt_workspace *ws, void *stream) {
    if (!ws) return fail(DBT_EINVAL, "workspace is NULL");
    DBT_CUDA(cudaMemsetAsync(ws->buf, 0, ws->L.total, (cudaStream_t)stream));
    return DBT_OK;
}

extern "C" dbt_status dbt_workspace_destroy(dbt_workspace *ws) {
    delete ws;
    return DBT_OK;
}

// ------------------------------------------------------------------ integration
static dbt_status check_pose(const double *pose, Pose *out) {
    if (!pose) return fail(DBT_EINVAL, "pose is NULL");
    for (int i = 0; i < 12; ++i)
        if (!std::isfinite(pose[i])) return fail(DBT_EINVAL, "pose has a non-finite entry");
    double R[9];
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) R[3 * r + c] = pose[4 * r + c];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double dot = 0.0;
            for (int c = 0; c < 3; ++c) dot += R[3 * i + c] * R[3 * j + c];
            if (std::fabs(dot - (i == j ? 1.0 : 0.0)) > 1e-6)
                return fail(DBT_EINVAL, "pose rotation is not orthonormal");
        }
    const double det = R[0] * (R[4] * R[8] - R[5] * R[7]) - R[1] * (R[3] * R[8] - R[5] * R[6]) +
                       R[2] * (R[3] * R[7] - R[4] * R[6]);
    if (!(det > 0.0)) return fail(DBT_EINVAL, "pose rotation has det <= 0");
    for (int i = 0; i < 9; ++i) out->r[i] = R[i];
    for (int r = 0; r < 3; ++r) out->t[r] = pose[4 * r + 3];
    return DBT_OK;
}

// Binary32 filter data of a pose for one grid.  b = (t - origin) * inv_res is
// taken in binary64 and split into an integer B and a remainder |b - B| <=
// 1/2, so that the binary32 coordinate fa . p + fb stays small; fe0 covers
// the rounding of fb (<= 2^-25) and of the binary64 path's own additions
// (<= 2^-50 (|t| + |origin|) inv_res), both with a wide margin.
void dbt::pose_filter(Pose &P, const DevGrid &g) {
    P.fast = 0;
    const double org[3] = {g.ox, g.oy, g.oz};
    for (int r = 0; r < 3; ++r) {
        const double b = (P.t[r] - org[r]) * g.inv_res;
        if (!(std::fabs(b) < 1e9)) return;
        const double B = std::round(b);
        P.fbi[r] = (int)B;
        P.fb[r] = (float)(b - B);
        P.fe0[r] = (float)((std::fabs(P.t[r]) + std::fabs(org[r])) * g.inv_res * 0x1p-46 + 0x1p-22);
        for (int j = 0; j < 3; ++j) {
            const double a = P.r[3 * r + j] * g.inv_res;
            if (!(std::fabs(a) < 1e30)) return;
            P.fa[3 * r + j] = (float)a;
            P.fr[3 * r + j] = (float)P.r[3 * r + j];
        }
    }
    P.fast = 1;
}

static dbt_status enqueue_prep(const dbt_grid *g, const dbt_kernels *k, dbt_workspace *ws,
                               const float *d_xyz, int64_t n, const double pose[12],
                               cudaStream_t s, DevGrid *dg_out, uint32_t *hcap_out,
                               const dbt_scan_options *opt = nullptr);

// Counters for pinned (device-mapped, 8-byte aligned) host memory are
// stored by the integrate kernel that publishes them, so no copy sits between
// one scan's kernels and the next scan's; null for other memory, which gets
// a copy on the stream.
static ScanStats *mapped_stats(dbt_scan_stats *h_stats) {
    if (!h_stats) return nullptr;
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, h_stats) != cudaSuccess) {
        (void)cudaGetLastError();                      // this query's own error only
        return nullptr;
    }
    if (a.type == cudaMemoryTypeHost && a.devicePointer &&
        (reinterpret_cast<uintptr_t>(a.devicePointer) & 7u) == 0u)
        return static_cast<ScanStats *>(a.devicePointer);
    return nullptr;
}

static dbt_status enqueue_scan(const dbt_grid *g, const dbt_kernels *k, dbt_workspace *ws,
                               const float *d_xyz, int64_t n, const double pose[12],
                               cudaStream_t s, const dbt_scan_options *opt = nullptr) {
    DevGrid dg;
    uint32_t hcap;
    dbt_status st = enqueue_prep(g, k, ws, d_xyz, n, pose, s, &dg, &hcap, opt);
    if (st != DBT_OK) return st;
    const int ni = (int)n;
    launch_alloc(dg, k->dp, n, ws->d, hcap, s);
    launch_fill(dg, k->dp, ni, ws->d, hcap, s);
    if (ws->ev_begin) DBT_CUDA(cudaEventRecord(ws->ev_begin, s));
    launch_integrate(dg, k->dp, k->dt, (long long)n, ws->d,
                     ws->ctas ? ws->ctas : integrate_grid_ctas(k->dp, ws->bz), s);
    if (ws->ev_end) DBT_CUDA(cudaEventRecord(ws->ev_end, s));
    DBT_CUDA(cudaGetLastError());
    return DBT_OK;
}

// Checks the arguments and enqueues the per-return stages that every scan
// starts with (transform, voxel, bin, first-return rule, brick counts).
static dbt_status enqueue_prep(const dbt_grid *g, const dbt_kernels *k, dbt_workspace *ws,
                               const float *d_xyz, int64_t n, const double pose[12],
                               cudaStream_t s, DevGrid *dg_out, uint32_t *hcap_out,
                               const dbt_scan_options *opt) {
    if (!k) return fail(DBT_EINVAL, "kernels is NULL");
    if (!ws) return fail(DBT_EINVAL, "workspace is NULL");
    dbt_status st = check_grid(g);
    if (st != DBT_OK) return st;
    if (g->nx != ws->nx || g->ny != ws->ny || g->nz != ws->nz || g->pitch_x != ws->pitch)
        return fail(DBT_EINVAL, "grid geometry differs from the workspace's");
    if (k->dp.K != ws->K) return fail(DBT_EINVAL, "kernel size differs from the workspace's");
    if (n < 0 || n > ws->max_points)
        return fail(DBT_EINVAL, "n = %lld outside [0, max_points = %lld]", (long long)n, ws->max_points);
    if (n > 0 && (!d_xyz || ((uintptr_t)d_xyz & 3u)))
        return fail(DBT_EINVAL, "points must be a non-NULL 4-byte aligned device pointer");
    const DevGrid dg = dev_grid(g, ws->bz);
    Pose P{};
    ScanEx ex{1, 0, 1};
    const bool use_ex = opt != nullptr;
    if (use_ex) {
        if (opt->downsample < 1) return fail(DBT_EINVAL, "downsample must be >= 1");
        if (opt->n_poses < 0 || opt->n_poses > MAX_SCAN_POSES)
            return fail(DBT_EINVAL, "n_poses must be in [0, %d]", MAX_SCAN_POSES);
        if (opt->n_poses > 0 && (!opt->poses || opt->period < 1))
            return fail(DBT_EINVAL, "motion compensation needs poses and period >= 1");
        ex.ds = opt->downsample;
        ex.n_poses = opt->n_poses;
        ex.period = opt->n_poses > 0 ? opt->period : 1;
        if (opt->n_poses > 0) {
            Pose table[MAX_SCAN_POSES];
            for (int m = 0; m < opt->n_poses; ++m) {
                st = check_pose(opt->poses + 12 * m, &table[m]);
                if (st != DBT_OK) return st;
                pose_filter(table[m], dg);
            }
            DBT_CUDA(cudaMemcpyAsync(ws->d.poses, table, sizeof(Pose) * opt->n_poses,
                                     cudaMemcpyHostToDevice, s));
        } else {
            st = check_pose(pose, &P);
            if (st != DBT_OK) return st;
        }
    } else {
        st = check_pose(pose, &P);
        if (st != DBT_OK) return st;
    }
    pose_filter(P, dg);
    uint32_t hcap = 64;
    while (hcap < 2ull * (unsigned long long)n) hcap <<= 1;
    const int ni = (int)n;
    launch_voxelize(dg, k->dp, k->dt, P, d_xyz, ni, ws->d, hcap, s, use_ex ? &ex : nullptr);
    *dg_out = dg;
    *hcap_out = hcap;
    return DBT_OK;
}

extern "C" dbt_status dbt_scan_contacts(const dbt_grid *g, const dbt_kernels *k, const float *d_xyz,
                                        int64_t n, const double pose[12], int32_t *d_out,
                                        void *stream) {
    if (!k) return fail(DBT_EINVAL, "kernels is NULL");
    dbt_status st = check_grid(g);
    if (st != DBT_OK) return st;
    if (n < 0 || n > (int64_t)1 << 40) return fail(DBT_EINVAL, "n = %lld out of range", (long long)n);
    if (n > 0 && (!d_xyz || ((uintptr_t)d_xyz & 3u)))
        return fail(DBT_EINVAL, "points must be a non-NULL 4-byte aligned device pointer");
    if (n > 0 && (!d_out || ((uintptr_t)d_out & 15u)))
        return fail(DBT_EINVAL, "out must be a non-NULL 16-byte aligned device pointer");
    Pose P{};
    st = check_pose(pose, &P);
    if (st != DBT_OK) return st;
    const DevGrid dg = dev_grid(g);
    pose_filter(P, dg);
    launch_contacts(dg, k->dp, k->dt, P, d_xyz, (long long)n, (int4 *)d_out, (cudaStream_t)stream);
    DBT_CUDA(cudaGetLastError());
    return DBT_OK;
}

extern "C" dbt_status dbt_workspace_set_timing(dbt_workspace *ws, void *ev_begin, void *ev_end) {
    if (!ws) return fail(DBT_EINVAL, "workspace is NULL");
    ws->ev_begin = (cudaEvent_t)ev_begin;
    ws->ev_end = (cudaEvent_t)ev_end;
    return DBT_OK;
}

extern "C" dbt_status dbt_scan_footprint(const dbt_grid *g, const dbt_kernels *k, dbt_workspace *ws,
                                         const float *d_xyz, int64_t n, const double pose[12],
                                         void *d_bits, size_t bits_bytes, int64_t h_counts[2],
                                         void *stream) {
    if (!h_counts) return fail(DBT_EINVAL, "h_counts is NULL");
    if (!g) return fail(DBT_EINVAL, "grid is NULL");
    const size_t words = ((size_t)g->pitch_x * g->ny * g->nz + 31) / 32;
    if (!d_bits || bits_bytes < 2 * words * 4 + 16)
        return fail(DBT_EINVAL, "footprint buffer needs %zu bytes", 2 * words * 4 + 16);
    cudaStream_t s = (cudaStream_t)stream;
    DevGrid dg;
    uint32_t hcap;
    dbt_status st = enqueue_prep(g, k, ws, d_xyz, n, pose, s, &dg, &hcap);
    if (st != DBT_OK) return st;
    uint32_t *bits_u = (uint32_t *)d_bits;
    uint32_t *bits_s = bits_u + words;
    unsigned long long *counts = (unsigned long long *)(bits_s + words);
    DBT_CUDA(cudaMemsetAsync(d_bits, 0, 2 * words * 4 + 16, s));
    launch_footprint(dg, k->dp, k->dt, (int)n, ws->d, hcap, bits_u, bits_s, counts, s);
    DBT_CUDA(cudaGetLastError());
    unsigned long long c[2];
    DBT_CUDA(cudaMemcpyAsync(c, counts, sizeof c, cudaMemcpyDeviceToHost, s));
    DBT_CUDA(cudaStreamSynchronize(s));
    h_counts[0] = (int64_t)c[0];
    h_counts[1] = (int64_t)c[1];
    return DBT_OK;
}

extern "C" dbt_status dbt_integrate_scan(const dbt_grid *g, const dbt_kernels *k, dbt_workspace *ws,
                                         const float *d_xyz, int64_t n, const double pose[12],
                                         void *stream) {
    return enqueue_scan(g, k, ws, d_xyz, n, pose, (cudaStream_t)stream);
}

extern "C" dbt_status dbt_integrate_scan_ex(const dbt_grid *g, const dbt_kernels *k,
                                            dbt_workspace *ws, const float *d_xyz, int64_t n,
                                            const double pose[12], const dbt_scan_options *opt,
                                            void *stream) {
    if (!opt) return enqueue_scan(g, k, ws, d_xyz, n, pose, (cudaStream_t)stream);
    return enqueue_scan(g, k, ws, d_xyz, n, pose, (cudaStream_t)stream, opt);
}

// Motion-compensation pose at time fraction tau between T0 and T1.  Full:
// R0 Exp(tau Log(R0^T R1)) (Rodrigues), yaw-only: Rz(tau dpsi) R0 with the
// yaw difference wrapped into (-pi, pi]; translation linear in both.
static void pose_at(const double *T0, const double *T1, double tau, int mode, double *out) {
    double R0[9], R1[9], Q[9];
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) {
            R0[3 * r + c] = T0[4 * r + c];
            R1[3 * r + c] = T1[4 * r + c];
        }
    if (mode == DBT_MOTION_YAW) {
        double dpsi = std::atan2(R1[3], R1[0]) - std::atan2(R0[3], R0[0]);
        while (dpsi > kPi) dpsi -= 2.0 * kPi;
        while (dpsi <= -kPi) dpsi += 2.0 * kPi;
        const double a = tau * dpsi, ca = std::cos(a), sa = std::sin(a);
        for (int c = 0; c < 3; ++c) {
            Q[c] = ca * R0[c] - sa * R0[3 + c];
            Q[3 + c] = sa * R0[c] + ca * R0[3 + c];
            Q[6 + c] = R0[6 + c];
        }
    } else {
        double D[9];
        for (int r = 0; r < 3; ++r)
            for (int c = 0; c < 3; ++c)
                D[3 * r + c] = R0[r] * R1[c] + R0[3 + r] * R1[3 + c] + R0[6 + r] * R1[6 + c];
        const double cth = std::min(1.0, std::max(-1.0, (D[0] + D[4] + D[8] - 1.0) / 2.0));
        const double th = std::acos(cth);
        double w[3] = {0.0, 0.0, 0.0};
        if (th > 1e-12) {
            if (th < kPi - 1e-6) {
                const double f = 1.0 / (2.0 * std::sin(th));
                w[0] = (D[7] - D[5]) * f;
                w[1] = (D[2] - D[6]) * f;
                w[2] = (D[3] - D[1]) * f;
            } else {   // half turn: D ~ 2 w w^T - I
                int j = 0;
                for (int a = 1; a < 3; ++a)
                    if (D[4 * a] > D[4 * j]) j = a;
                for (int a = 0; a < 3; ++a) w[a] = D[3 * a + j] + (a == j ? 1.0 : 0.0);
                const int j1 = (j + 1) % 3, j2 = (j + 2) % 3;
                const double sg = (D[3 * j2 + j1] - D[3 * j1 + j2]) < 0.0 ? -1.0 : 1.0;
                const double nw = std::sqrt(w[0] * w[0] + w[1] * w[1] + w[2] * w[2]);
                for (int a = 0; a < 3; ++a) w[a] = sg * w[a] / nw;
            }
        }
        const double phi = tau * th, s = std::sin(phi), c1 = 1.0 - std::cos(phi);
        const double K[9] = {0.0, -w[2], w[1], w[2], 0.0, -w[0], -w[1], w[0], 0.0};
        double E[9];
        for (int r = 0; r < 3; ++r)
            for (int c = 0; c < 3; ++c) {
                const double kk = K[3 * r] * K[c] + K[3 * r + 1] * K[3 + c] + K[3 * r + 2] * K[6 + c];
                E[3 * r + c] = (r == c ? 1.0 : 0.0) + s * K[3 * r + c] + c1 * kk;
            }
        for (int r = 0; r < 3; ++r)
            for (int c = 0; c < 3; ++c)
                Q[3 * r + c] = R0[3 * r] * E[c] + R0[3 * r + 1] * E[3 + c] + R0[3 * r + 2] * E[6 + c];
    }
    for (int r = 0; r < 3; ++r) {
        for (int c = 0; c < 3; ++c) out[4 * r + c] = Q[3 * r + c];
        out[4 * r + 3] = T0[4 * r + 3] + tau * (T1[4 * r + 3] - T0[4 * r + 3]);
    }
}

extern "C" dbt_status dbt_pose_ramp(const double start[12], const double end[12], int32_t n_poses,
                                    int32_t mode, double *out) {
    if (!start || !end || !out) return fail(DBT_EINVAL, "NULL argument");
    if (n_poses < 1 || n_poses > MAX_SCAN_POSES)
        return fail(DBT_EINVAL, "n_poses must be in [1, %d]", MAX_SCAN_POSES);
    if (mode != DBT_MOTION_FULL && mode != DBT_MOTION_YAW) return fail(DBT_EINVAL, "unknown mode");
    Pose tmp;
    dbt_status st = check_pose(start, &tmp);
    if (st == DBT_OK) st = check_pose(end, &tmp);
    if (st != DBT_OK) return st;
    for (int m = 0; m < n_poses; ++m)
        pose_at(start, end, ((double)m + 0.5) / (double)n_poses, mode, out + 12 * m);
    return DBT_OK;
}

// One scan on a scratch buffer owned by the caller of this function (the
// no-allocation entry point): a workspace view lives on the stack, the
// regions that must start at zero are cleared on the stream, and nothing is
// allocated on the host or the device.
dbt_status dbt::report_einval(const char *msg) { return fail(DBT_EINVAL, "%s", msg); }

dbt_status dbt::scratch_fits(int32_t pitch_x, int32_t ny, int32_t nz, int32_t K, int64_t n,
                             size_t bytes, long long max_points) {
    if (K < 1 || K > MAX_K || (K % 2) == 0)
        return fail(DBT_EINVAL, "kernel_size must be odd and in [1, %d]", MAX_K);
    if (pitch_x < 32 || (pitch_x % 32) != 0 || ny < 1 || nz < 1)
        return fail(DBT_EINVAL, "grid dims must be >= 1 (pitch a multiple of 32)");
    if (n < 0 || n > max_points)
        return fail(DBT_EINVAL, "n = %lld exceeds the no-allocation limit of %lld returns per scan",
                    (long long)n, max_points);
    WsLayout L;
    dbt_status st = ws_layout_dims(pitch_x, ny, nz, K, max_points, &L, false, BZ_DEFAULT);
    if (st != DBT_OK) return st;
    if (L.total > bytes)
        return fail(DBT_EINVAL,
                    "grid too large for the no-allocation scratch: needs %zu bytes, limit %zu "
                    "(%u bricks of 32x8x8 voxels)", L.total, bytes, L.nbricks);
    return DBT_OK;
}

dbt_status dbt::scratch_fits_grid(const dbt_grid *g, const dbt_kernels *k, int64_t n, size_t bytes,
                                  long long max_points) {
    if (!k) return fail(DBT_EINVAL, "kernels is NULL");
    dbt_status st = check_grid(g);
    if (st != DBT_OK) return st;
    return scratch_fits(g->pitch_x, g->ny, g->nz, k->dp.K, n, bytes, max_points);
}

dbt_status dbt::integrate_on_scratch(const dbt_grid *g, const dbt_kernels *k, const float *d_xyz,
                                     int64_t n, const double pose[12], void *scratch,
                                     size_t scratch_bytes, long long max_points,
                                     dbt_scan_stats *h_stats, cudaStream_t s) {
    dbt_status st = scratch_fits_grid(g, k, n, scratch_bytes, max_points);
    if (st != DBT_OK) return st;
    if (!scratch) return fail(DBT_EINVAL, "scratch is NULL");
    WsLayout L;
    st = ws_layout(g, k, max_points, &L, false, BZ_DEFAULT);   // the default depth only
    if (st != DBT_OK) return st;
    dbt_workspace w;
    st = ws_bind(&w, g, k, max_points, L, scratch);
    if (st != DBT_OK) return st;
    char *base = (char *)scratch;
    DBT_CUDA(cudaMemsetAsync(base + L.hdr, 0, up256(sizeof(WsHeader)), s));
    DBT_CUDA(cudaMemsetAsync(base + L.hkey, 0, L.bcnt - L.hkey, s));        // hash keys + indices
    DBT_CUDA(cudaMemsetAsync(base + L.bcnt, 0, (size_t)L.nbricks * 4, s));  // brick counters
    ScanStats *mapped = mapped_stats(h_stats);
    w.d.stats_out = mapped;
    st = enqueue_scan(g, k, &w, d_xyz, n, pose, s);
    if (st != DBT_OK) return st;
    if (h_stats && !mapped)
        DBT_CUDA(cudaMemcpyAsync(h_stats, &w.d.hdr->last, sizeof(dbt_scan_stats),
                                 cudaMemcpyDeviceToHost, s));
    return DBT_OK;
}

// ------------------------------------------------------------------ batches
// The grid views and brick bases of every brick depth live in the batch's
// buffer side by side (depth index 0, 1, 2 = 4, 8, 16), so a tuning changes
// the depth by pointing the launch at another set: nothing is written to the
// device, and a captured graph keeps the set it was captured with.
constexpr int N_DEPTHS = 3;
static int depth_index(int bz) { return bz_shift(bz) - 2; }

struct dbt_batch {
    const dbt_kernels *k = nullptr;
    int n_grids = 0;
    std::vector<DevGrid> grids;          // host copies at the default depth
    std::vector<dbt_grid> cgrids;
    std::vector<uint32_t> bbase;         // per depth n_grids + 1
    long long max_points = 0;
    int max_items = 0;
    WsLayout L;                          // integration scratch (bricks of all grids)
    WsDev d;
    void *buf = nullptr;
    size_t off_grids = 0, off_bbase = 0, off_items = 0, off_istart = 0, off_icnt = 0, total = 0;
    std::vector<ItemDev> items;          // staged descriptors of the current set
    std::vector<long long> istart;
    int n_items = 0;
    long long n_total = 0;
    BatchDev bd;
    int ctas = 0;                        // integrate grid; 0 = occupancy maximum
    int bz = BZ_DEFAULT;                 // brick depth
};

// Points the batch's launches at the grid views and brick bases of depth bz.
static void batch_use_depth(dbt_batch *b, int bz) {
    const int d = depth_index(bz);
    char *base = (char *)b->buf;
    b->bz = bz;
    b->bd.grids = (const DevGrid *)(base + b->off_grids) + (size_t)d * b->n_grids;
    b->bd.bbase = (const uint32_t *)(base + b->off_bbase) + (size_t)d * (b->n_grids + 1);
    b->bd.bzs = bz_shift(bz);
    b->d.nbricks = b->bbase[(size_t)d * (b->n_grids + 1) + b->n_grids];
}

static dbt_status batch_layout(const dbt_grid *grids, int n_grids, const dbt_kernels *k,
                               long long max_points, int max_items, WsLayout *L,
                               std::vector<uint32_t> *bbase, size_t *tail_offs /* 5 + total */) {
    if (!grids || n_grids < 1 || n_grids > MAX_BATCH_GRIDS)
        return fail(DBT_EINVAL, "n_grids must be in [1, %d]", MAX_BATCH_GRIDS);
    if (max_items < 1 || max_items > MAX_BATCH_ITEMS)
        return fail(DBT_EINVAL, "max_items must be in [1, %d]", MAX_BATCH_ITEMS);
    if (max_points < 1 || max_points > (1ll << 31) - 1)
        return fail(DBT_EINVAL, "max_points must be in [1, 2^31 - 1]");
    for (int m = 0; m < n_grids; ++m) {
        dbt_status st = check_grid(&grids[m]);
        if (st != DBT_OK) return fail(st, "grid %d: %s", m, dbt_last_error());
    }
    bbase->assign((size_t)N_DEPTHS * (n_grids + 1), 0u);
    unsigned long long nb = 0;                    // bricks at the shallowest depth: the most
    for (int d = N_DEPTHS - 1; d >= 0; --d) {
        uint32_t *bb = bbase->data() + (size_t)d * (n_grids + 1);
        nb = 0;
        for (int m = 0; m < n_grids; ++m) {
            bb[m] = (uint32_t)nb;
            nb += bricks_of(grids[m].pitch_x, grids[m].ny, grids[m].nz, 4 << d);
            if (nb >= (1ull << 32)) return fail(DBT_EINVAL, "too many bricks over the batch's grids");
        }
        bb[n_grids] = (uint32_t)nb;
    }
    // the single-grid layout with the batch's total brick count
    uint32_t hc = 64;
    while (hc < 2ull * (unsigned long long)max_points) hc <<= 1;
    L->nbricks = (uint32_t)nb;
    L->hcap_alloc = hc;
    L->pairs_cap = (unsigned long long)max_points * max_pairs_per_return(k->dp.K, BZ_MIN);
    L->max_touched = (uint32_t)std::min<unsigned long long>(nb, L->pairs_cap);
    size_t o = 0;
    L->hdr = o;      o += up256(sizeof(WsHeader));
    L->stage = o;    o += up256(16);
    L->stage_b = o;  o += up256(16);
    L->prec = o;     o += up256((size_t)max_points * 16);
    L->hkey = o;     o += up256((size_t)hc * 8);
    L->hidx = o;     o += up256((size_t)hc * 4);
    L->bcnt = o;     o += up256((size_t)nb * 4);
    L->boff = o;     o += up256((size_t)nb * 4);
    L->order = o;    o += up256((size_t)L->max_touched * 4);
    L->lq0 = o;      o += up256((size_t)L->max_touched * 4);
    L->lq1 = o;      o += up256((size_t)L->max_touched * 4);
    L->lq2 = o;      o += up256((size_t)L->max_touched * 4);
    L->pairs = o;    o += up256((size_t)L->pairs_cap * 4);
    L->poses = o;    o += up256((size_t)MAX_SCAN_POSES * sizeof(Pose));
    L->total = o;
    tail_offs[0] = o;  o += up256((size_t)N_DEPTHS * n_grids * sizeof(DevGrid));
    tail_offs[1] = o;  o += up256((size_t)N_DEPTHS * (n_grids + 1) * 4);
    tail_offs[2] = o;  o += up256((size_t)max_items * sizeof(ItemDev));
    tail_offs[3] = o;  o += up256((size_t)(max_items + 1) * 8);
    tail_offs[4] = o;  o += up256((size_t)max_items * sizeof(ItemCounters));
    tail_offs[5] = o;
    return DBT_OK;
}

extern "C" dbt_status dbt_batch_size(const dbt_grid *grids, int32_t n_grids, const dbt_kernels *k,
                                     int64_t max_points, int32_t max_items, size_t *bytes) {
    if (!k) return fail(DBT_EINVAL, "kernels is NULL");
    if (!bytes) return fail(DBT_EINVAL, "bytes is NULL");
    WsLayout L;
    std::vector<uint32_t> bb;
    size_t offs[6];
    dbt_status st = batch_layout(grids, n_grids, k, max_points, max_items, &L, &bb, offs);
    if (st != DBT_OK) return st;
    *bytes = offs[5];
    return DBT_OK;
}

extern "C" dbt_status dbt_batch_create(const dbt_grid *grids, int32_t n_grids, const dbt_kernels *k,
                                       int64_t max_points, int32_t max_items, void *d_buf,
                                       size_t bytes, void *stream, dbt_batch **out) {
    if (!out) return fail(DBT_EINVAL, "out is NULL");
    *out = nullptr;
    if (!k) return fail(DBT_EINVAL, "kernels is NULL");
    if (!d_buf || !aligned256(d_buf)) return fail(DBT_EINVAL, "batch buffer must be 256-byte aligned");
    dbt_batch *b = new (std::nothrow) dbt_batch();
    if (!b) return fail(DBT_ENOMEM, "host allocation failed");
    size_t offs[6];
    dbt_status st = batch_layout(grids, n_grids, k, max_points, max_items, &b->L, &b->bbase, offs);
    if (st != DBT_OK) {
        delete b;
        return st;
    }
    if (bytes < offs[5]) {
        delete b;
        return fail(DBT_ENOMEM, "batch buffer too small: %zu < %zu bytes", bytes, offs[5]);
    }
    b->k = k;
    b->n_grids = n_grids;
    b->max_points = max_points;
    b->max_items = max_items;
    b->buf = d_buf;
    b->off_grids = offs[0];
    b->off_bbase = offs[1];
    b->off_items = offs[2];
    b->off_istart = offs[3];
    b->off_icnt = offs[4];
    b->total = offs[5];
    for (int m = 0; m < n_grids; ++m) {
        b->grids.push_back(dev_grid(&grids[m]));
        b->cgrids.push_back(grids[m]);
    }
    char *base = (char *)d_buf;
    dbt_workspace w;
    dbt_status bst = ws_bind(&w, &grids[0], k, max_points, b->L, d_buf);
    if (bst != DBT_OK) {
        delete b;
        return bst;
    }
    b->d = w.d;
    std::vector<DevGrid> views;                  // every depth's grid views, depth-major
    for (int d = 0; d < N_DEPTHS; ++d)
        for (int m = 0; m < n_grids; ++m) views.push_back(dev_grid(&grids[m], 4 << d));
    batch_use_depth(b, BZ_DEFAULT);
    b->bd.items = (const ItemDev *)(base + b->off_items);
    b->bd.istart = (const long long *)(base + b->off_istart);
    b->bd.icnt = (ItemCounters *)(base + b->off_icnt);
    b->bd.n_grids = n_grids;
    b->bd.n_items = 0;
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaMemsetAsync(d_buf, 0, b->total, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(base + b->off_grids, views.data(), views.size() * sizeof(DevGrid),
                            cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(base + b->off_bbase, b->bbase.data(), b->bbase.size() * 4,
                            cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        delete b;
        return cuda_fail(e, "batch set-up");
    }
    *out = b;
    return DBT_OK;
}

extern "C" dbt_status dbt_batch_set_items(dbt_batch *b, const dbt_batch_item *items, int32_t n_items,
                                          void *stream) {
    if (!b) return fail(DBT_EINVAL, "batch is NULL");
    if (n_items < 0 || n_items > b->max_items)
        return fail(DBT_EINVAL, "n_items = %d outside [0, %d]", n_items, b->max_items);
    if (n_items > 0 && !items) return fail(DBT_EINVAL, "items is NULL");
    b->items.resize(std::max(1, n_items));
    b->istart.assign(n_items + 1, 0ll);
    long long total = 0;
    for (int i = 0; i < n_items; ++i) {
        const dbt_batch_item &it = items[i];
        if (it.grid < 0 || it.grid >= b->n_grids)
            return fail(DBT_EINVAL, "item %d: grid %d outside [0, %d)", i, it.grid, b->n_grids);
        if (it.n < 0) return fail(DBT_EINVAL, "item %d: n < 0", i);
        if (it.n > 0 && (!it.d_xyz || ((uintptr_t)it.d_xyz & 3u)))
            return fail(DBT_EINVAL, "item %d: points must be a 4-byte aligned device pointer", i);
        Pose P;
        dbt_status st = check_pose(it.pose, &P);
        if (st != DBT_OK) return fail(st, "item %d: %s", i, dbt_last_error());
        pose_filter(P, b->grids[it.grid]);
        ItemDev &d = b->items[i];
        d.xyz = it.d_xyz;
        d.n = it.n;
        d.grid = it.grid;
        d.pad = 0;
        d.pose = P;
        b->istart[i] = total;
        total += it.n;
        if (total > b->max_points)
            return fail(DBT_EINVAL, "the items hold more than max_points = %lld returns", b->max_points);
    }
    b->istart[n_items] = total;
    char *base = (char *)b->buf;
    cudaStream_t s = (cudaStream_t)stream;
    // pageable sources: each copy waits for earlier work on the stream, so a
    // running batch never sees its descriptors change
    if (n_items > 0)
        DBT_CUDA(cudaMemcpyAsync(base + b->off_items, b->items.data(), n_items * sizeof(ItemDev),
                                 cudaMemcpyHostToDevice, s));
    DBT_CUDA(cudaMemcpyAsync(base + b->off_istart, b->istart.data(), (n_items + 1) * 8,
                             cudaMemcpyHostToDevice, s));
    b->n_items = n_items;
    b->n_total = total;
    b->bd.n_items = n_items;
    return DBT_OK;
}

extern "C" dbt_status dbt_batch_run(dbt_batch *b, void *stream) {
    if (!b) return fail(DBT_EINVAL, "batch is NULL");
    cudaStream_t s = (cudaStream_t)stream;
    const dbt_kernels *k = b->k;
    uint32_t hcap = 64;
    while (hcap < 2ull * (unsigned long long)b->n_total) hcap <<= 1;
    if (b->n_items > 0)
        DBT_CUDA(cudaMemsetAsync((char *)b->buf + b->off_icnt, 0, b->n_items * sizeof(ItemCounters), s));
    if (b->n_items > 0) {
        launch_voxelize_batch(b->bd, k->dp, k->dt, b->n_total, b->d, hcap, s);
    }
    launch_alloc_batch(b->bd, k->dp, b->n_total, b->d, hcap, s);
    if (b->n_items > 0) launch_fill_batch(b->bd, k->dp, b->n_total, b->d, hcap, s);
    launch_integrate_batch(b->bd, k->dp, k->dt, b->n_total, b->d,
                           b->ctas ? b->ctas : integrate_grid_ctas(k->dp, b->bz), s);
    DBT_CUDA(cudaGetLastError());
    return DBT_OK;
}

// ------------------------------------------------------------------ tuning
// Brick depth of a tuning (0 = the default).
static int tuning_depth(const dbt_tuning *t) { return t->brick_depth ? t->brick_depth : BZ_DEFAULT; }

static dbt_status check_tuning(const dbt_tuning *t, const dbt_kernels *k) {
    if (!t) return fail(DBT_EINVAL, "tuning is NULL");
    if (t->heavy_pairs < 0) return fail(DBT_EINVAL, "heavy_pairs must be >= 0");
    const int bz = tuning_depth(t);
    if (bz != 4 && bz != 8 && bz != 16) return fail(DBT_EINVAL, "brick_depth must be 0, 4, 8 or 16");
    if (bz == 16 && k->dp.K > BZ16_MAX_K)
        return fail(DBT_EINVAL, "brick_depth 16 needs kernel_size <= %d", BZ16_MAX_K);
    const int cap = 4 * integrate_grid_ctas(k->dp, bz);
    if (t->integrate_ctas < 0 || t->integrate_ctas > cap)
        return fail(DBT_EINVAL, "integrate_ctas must be in [0, %d]", cap);
    return DBT_OK;
}

extern "C" dbt_status dbt_workspace_set_tuning(dbt_workspace *ws, const dbt_kernels *k,
                                               const dbt_tuning *t) {
    if (!ws || !k) return fail(DBT_EINVAL, "workspace or kernels is NULL");
    dbt_status st = check_tuning(t, k);
    if (st != DBT_OK) return st;
    const int bz = tuning_depth(t);
    const unsigned long long nb = bricks_of(ws->pitch, ws->ny, ws->nz, bz);
    if (nb > ws->L.nbricks || (unsigned long long)ws->max_points * max_pairs_per_return(ws->K, bz) >
                                  ws->L.pairs_cap)
        return fail(DBT_EINVAL, "the workspace has no room for bricks of depth %d", bz);
    ws->d.heavy = (uint32_t)t->heavy_pairs;
    ws->ctas = t->integrate_ctas;
    ws->bz = bz;
    ws->d.nbricks = (uint32_t)nb;
    return DBT_OK;
}

extern "C" dbt_status dbt_workspace_get_tuning(const dbt_workspace *ws, dbt_tuning *t) {
    if (!ws || !t) return fail(DBT_EINVAL, "NULL argument");
    t->heavy_pairs = (int32_t)ws->d.heavy;
    t->integrate_ctas = ws->ctas;
    t->brick_depth = ws->bz;
    return DBT_OK;
}

extern "C" dbt_status dbt_batch_set_tuning(dbt_batch *b, const dbt_tuning *t) {
    if (!b) return fail(DBT_EINVAL, "batch is NULL");
    dbt_status st = check_tuning(t, b->k);
    if (st != DBT_OK) return st;
    b->d.heavy = (uint32_t)t->heavy_pairs;
    b->ctas = t->integrate_ctas;
    batch_use_depth(b, tuning_depth(t));
    return DBT_OK;
}

extern "C" dbt_status dbt_batch_get_tuning(const dbt_batch *b, dbt_tuning *t) {
    if (!b || !t) return fail(DBT_EINVAL, "NULL argument");
    t->heavy_pairs = (int32_t)b->d.heavy;
    t->integrate_ctas = b->ctas;
    t->brick_depth = b->bz;
    return DBT_OK;
}

// Candidates, searched in two stages.  Stage 1: the brick depth (8, 4 and,
// up to K = 17, 16) crossed with the heavy threshold (CTA mode from 16 to
// 256 pairs per brick; the pairs a brick gets scale with its depth), on the
// occupancy-maximum grid.  Stage 2: the winner's depth and threshold on a
// persistent grid of three, two or one CTAs per SM.  Each candidate is
// timed over n_trials runs after one warm-up run.
static std::vector<dbt_tuning> depth_heavy_candidates(const dbt_kernels *k) {
    std::vector<dbt_tuning> out;
    for (int bz : {8, 4, 16}) {
        if (bz == 16 && k->dp.K > BZ16_MAX_K) continue;
        for (int h : {16, 24, 32, 40, 48, 64, 96, 128, 192, 256}) out.push_back(dbt_tuning{h, 0, bz});
    }
    return out;
}

static std::vector<dbt_tuning> grid_candidates(const dbt_kernels *k, const dbt_tuning &best) {
    const int sms = device_sm_count(), full = integrate_grid_ctas(k->dp, tuning_depth(&best));
    std::vector<dbt_tuning> out;
    for (int c : {3 * sms, 2 * sms, sms})
        if (c < full) out.push_back(dbt_tuning{best.heavy_pairs, c, best.brick_depth});
    return out;
}

template <typename Run>
static dbt_status time_candidates(const std::vector<dbt_tuning> &cands, int n_trials, cudaStream_t s,
                                  Run run, dbt_tuning *best, float *best_ms) {
    cudaEvent_t e0, e1;
    DBT_CUDA(cudaEventCreate(&e0));
    DBT_CUDA(cudaEventCreate(&e1));
    dbt_status st = DBT_OK;
    for (const dbt_tuning &c : cands) {
        if ((st = run(c)) != DBT_OK) break;                 // warm-up with this tuning
        cudaEventRecord(e0, s);
        for (int i = 0; i < n_trials && st == DBT_OK; ++i) st = run(c);
        cudaEventRecord(e1, s);
        if (st != DBT_OK) break;
        cudaError_t e = cudaEventSynchronize(e1);
        if (e != cudaSuccess) {
            st = cuda_fail(e, "cudaEventSynchronize(autotune)");
            break;
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < *best_ms) {
            *best_ms = ms;
            *best = c;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return st;
}

template <typename Run>
static dbt_status autotune(const dbt_kernels *k, int n_trials, cudaStream_t s, Run run,
                           dbt_tuning *best) {
    if (n_trials < 1 || n_trials > 1000) return fail(DBT_EINVAL, "n_trials must be in [1, 1000]");
    float best_ms = 3.4e38f;
    dbt_status st = time_candidates(depth_heavy_candidates(k), n_trials, s, run, best, &best_ms);
    if (st == DBT_OK) st = time_candidates(grid_candidates(k, *best), n_trials, s, run, best, &best_ms);
    return st;
}

extern "C" dbt_status dbt_batch_autotune(dbt_batch *b, int32_t n_trials, void *stream,
                                         dbt_tuning *best) {
    if (!b || !best) return fail(DBT_EINVAL, "NULL argument");
    cudaStream_t s = (cudaStream_t)stream;
    dbt_status st = autotune(b->k, n_trials, s, [&](const dbt_tuning &c) {
        dbt_status r = dbt_batch_set_tuning(b, &c);
        return r == DBT_OK ? dbt_batch_run(b, stream) : r;
    }, best);
    if (st != DBT_OK) return st;
    return dbt_batch_set_tuning(b, best);
}

extern "C" dbt_status dbt_workspace_autotune(const dbt_grid *g, const dbt_kernels *k,
                                             dbt_workspace *ws, const float *d_xyz, int64_t n,
                                             const double pose[12], int32_t n_trials, void *stream,
                                             dbt_tuning *best) {
    if (!ws || !k || !best) return fail(DBT_EINVAL, "NULL argument");
    cudaStream_t s = (cudaStream_t)stream;
    dbt_status st = autotune(k, n_trials, s, [&](const dbt_tuning &c) {
        dbt_status r = dbt_workspace_set_tuning(ws, k, &c);
        return r == DBT_OK ? enqueue_scan(g, k, ws, d_xyz, n, pose, s) : r;
    }, best);
    if (st != DBT_OK) return st;
    return dbt_workspace_set_tuning(ws, k, best);
}

extern "C" dbt_status dbt_batch_stats(const dbt_batch *b, dbt_scan_stats *per_item, int32_t n,
                                      dbt_scan_stats *total, void *stream) {
    if (!b) return fail(DBT_EINVAL, "batch is NULL");
    if (n < 0 || n > b->n_items) return fail(DBT_EINVAL, "n outside [0, n_items]");
    DBT_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
    dbt_scan_stats tot;
    DBT_CUDA(cudaMemcpy(&tot, &b->d.hdr->last, sizeof tot, cudaMemcpyDeviceToHost));
    if (total) *total = tot;
    if (per_item && n > 0) {
        std::vector<ItemCounters> c(n);
        DBT_CUDA(cudaMemcpy(c.data(), (char *)b->buf + b->off_icnt, n * sizeof(ItemCounters),
                            cudaMemcpyDeviceToHost));
        for (int i = 0; i < n; ++i) {
            dbt_scan_stats &o = per_item[i];
            o.n_input = b->istart[i + 1] - b->istart[i];
            o.n_valid = (long long)c[i].valid;
            o.n_inside = (long long)c[i].inside;
            o.n_kept = (long long)c[i].kept;
            o.n_pairs = 0;
            o.n_bricks = 0;
            o.error = tot.error;
            o.reserved = 0;
        }
    }
    if (tot.error) return fail(DBT_ESTATE, "device error bits 0x%x", tot.error);
    return DBT_OK;
}

extern "C" dbt_status dbt_batch_destroy(dbt_batch *b) {
    delete b;
    return DBT_OK;
}

extern "C" dbt_status dbt_integrate_scan_host(const dbt_grid *g, const dbt_kernels *k,
                                              dbt_workspace *ws, const float *h_xyz, int64_t n,
                                              const double pose[12], dbt_scan_stats *h_stats,
                                              void *stream) {
    if (!ws) return fail(DBT_EINVAL, "workspace is NULL");
    if (n < 0 || n > ws->max_points) return fail(DBT_EINVAL, "n outside [0, max_points]");
    if (n > 0 && !h_xyz) return fail(DBT_EINVAL, "h_xyz is NULL");
    if (!ws->stage_b) return fail(DBT_ESTATE, "workspace has no host staging");
    cudaStream_t s = (cudaStream_t)stream;
    // The scan's returns are copied on the workspace's copy stream into the
    // staging buffer the scan before last used, so the copy overlaps the
    // previous scan's kernels; the scan's kernels wait for the copy.
    if (!ws->copy_stream) {
        DBT_CUDA(cudaStreamCreateWithFlags(&ws->copy_stream, cudaStreamNonBlocking));
        for (int i = 0; i < 2; ++i) {
            DBT_CUDA(cudaEventCreateWithFlags(&ws->ev_copied[i], cudaEventDisableTiming));
            DBT_CUDA(cudaEventCreateWithFlags(&ws->ev_free[i], cudaEventDisableTiming));
        }
    }
    const int i = ws->stage_next;
    float *buf = i ? ws->stage_b : ws->d.stage;
    DBT_CUDA(cudaStreamWaitEvent(ws->copy_stream, ws->ev_free[i], 0));   // its last reader is done
    if (n > 0)
        DBT_CUDA(cudaMemcpyAsync(buf, h_xyz, (size_t)n * 12, cudaMemcpyHostToDevice, ws->copy_stream));
    DBT_CUDA(cudaEventRecord(ws->ev_copied[i], ws->copy_stream));
    DBT_CUDA(cudaStreamWaitEvent(s, ws->ev_copied[i], 0));
    ScanStats *mapped = mapped_stats(h_stats);
    ws->d.stats_out = mapped;
    dbt_status st = enqueue_scan(g, k, ws, buf, n, pose, s);
    ws->d.stats_out = nullptr;
    if (st != DBT_OK) return st;
    DBT_CUDA(cudaEventRecord(ws->ev_free[i], s));
    ws->stage_next = i ^ 1;
    if (h_stats && !mapped)
        DBT_CUDA(cudaMemcpyAsync(h_stats, &ws->d.hdr->last, sizeof(dbt_scan_stats),
                                 cudaMemcpyDeviceToHost, s));
    return DBT_OK;
}

extern "C" dbt_status dbt_get_scan_stats(const dbt_workspace *ws, dbt_scan_stats *out, void *stream) {
    if (!ws) return fail(DBT_EINVAL, "workspace is NULL");
    DBT_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
    dbt_scan_stats st;
    DBT_CUDA(cudaMemcpy(&st, &ws->d.hdr->last, sizeof st, cudaMemcpyDeviceToHost));
    if (out) *out = st;
    if (st.error) return fail(DBT_ESTATE, "device error bits 0x%x", st.error);
    return DBT_OK;
}

extern "C" dbt_status dbt_sync(void *stream, const dbt_workspace *ws) {
    DBT_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
    if (ws) {
        dbt_scan_stats st;
        DBT_CUDA(cudaMemcpy(&st, &ws->d.hdr->last, sizeof st, cudaMemcpyDeviceToHost));
        if (st.error) return fail(DBT_ESTATE, "device error bits 0x%x", st.error);
    }
    return DBT_OK;
}

// ------------------------------------------------------------------ readouts
extern "C" dbt_status dbt_bin_directions(const dbt_kernels *k, const double *d_dirs, int64_t n,
                                         int32_t *d_bins, void *stream) {
    if (!k) return fail(DBT_EINVAL, "kernels is NULL");
    if (n < 0 || n > 0x7FFFFFFF) return fail(DBT_EINVAL, "bad n");
    if (n > 0 && (!d_dirs || !d_bins)) return fail(DBT_EINVAL, "NULL buffer");
    launch_bin_dirs(k->dp, k->dt, d_dirs, (int)n, d_bins, (cudaStream_t)stream);
    DBT_CUDA(cudaGetLastError());
    return DBT_OK;
}

extern "C" dbt_status dbt_read_voxels(const dbt_grid *g, const int32_t *d_idx, int64_t n,
                                      uint32_t *d_mask, uint8_t *d_sign, uint16_t *d_hits,
                                      void *stream) {
    dbt_status st = check_grid(g);
    if (st != DBT_OK) return st;
    if (n < 0) return fail(DBT_EINVAL, "n < 0");
    if (n > 0 && !d_idx) return fail(DBT_EINVAL, "d_idx is NULL");
    launch_read_voxels(dev_grid(g), d_idx, n, d_mask, d_sign, d_hits, (cudaStream_t)stream);
    DBT_CUDA(cudaGetLastError());
    return DBT_OK;
}

extern "C" dbt_status dbt_read_distance(const dbt_grid *g, const int32_t *d_idx, int64_t n,
                                        float *d_sdf, void *stream) {
    dbt_status st = check_grid(g);
    if (st != DBT_OK) return st;
    if (n < 0) return fail(DBT_EINVAL, "n < 0");
    if (n > 0 && (!d_idx || !d_sdf)) return fail(DBT_EINVAL, "NULL buffer");
    launch_read_distance(dev_grid(g), g->res, d_idx, n, d_sdf, (cudaStream_t)stream);
    DBT_CUDA(cudaGetLastError());
    return DBT_OK;
}

// ------------------------------------------------------------------ export
static dbt_status export_box(const dbt_grid *g, const int32_t box[6], ExportBox *b) {
    if (!box) return fail(DBT_EINVAL, "box is NULL");
    for (int a = 0; a < 3; ++a) {
        const int n = a == 0 ? g->nx : a == 1 ? g->ny : g->nz;
        if (box[a] < 0 || box[a + 3] < 0 || (long long)box[a] + box[a + 3] > n)
            return fail(DBT_EINVAL, "box axis %d outside the grid", a);
    }
    b->x0 = box[0];
    b->y0 = box[1];
    b->z0 = box[2];
    b->bx = box[3];
    b->by = box[4];
    b->bz = box[5];
    b->cx = std::max(0, box[3] - 1);
    b->cy = std::max(0, box[4] - 1);
    b->cz = std::max(0, box[5] - 1);
    b->ncell = b->cx * b->cy * b->cz;
    return DBT_OK;
}

// Inside bits over (sign, popcount): bit s * 33 + p is f < iso with the
// mesh's binary32 field f = (s ? 1 : -1) * p * res (res, iso rounded to float).
static void inside_lut(double res, double iso, uint64_t *lut0, uint64_t *lut1) {
    *lut0 = 0;
    *lut1 = 0;
    const float resf = (float)res, isof = (float)iso;
    for (int s = 0; s < 2; ++s)
        for (int p = 0; p <= 32; ++p) {
            const float f = (s ? 1.0f : -1.0f) * (float)p * resf;
            if (f < isof) {
                const int idx = s * 33 + p;
                if (idx < 64) *lut0 |= 1ull << idx;
                else *lut1 |= 1ull << (idx - 64);
            }
        }
}

extern "C" dbt_status dbt_sdf_field(const dbt_grid *g, const int32_t box[6], float *d_out,
                                    void *stream) {
    dbt_status st = check_grid(g);
    if (st != DBT_OK) return st;
    ExportBox b;
    if ((st = export_box(g, box, &b)) != DBT_OK) return st;
    if ((long long)b.bx * b.by * b.bz > 0 && !d_out) return fail(DBT_EINVAL, "d_out is NULL");
    launch_sdf_field(dev_grid(g), g->res, b, d_out, (cudaStream_t)stream);
    DBT_CUDA(cudaGetLastError());
    return DBT_OK;
}

extern "C" dbt_status dbt_mesh_scratch_size(const dbt_grid *g, const int32_t box[6],
                                            size_t *bytes) {
    dbt_status st = check_grid(g);
    if (st != DBT_OK) return st;
    ExportBox b;
    if ((st = export_box(g, box, &b)) != DBT_OK) return st;
    if (!bytes) return fail(DBT_EINVAL, "bytes is NULL");
    *bytes = mc_scratch_bytes(b);
    return DBT_OK;
}

extern "C" dbt_status dbt_mesh_extract(const dbt_grid *g, const int32_t box[6], double iso,
                                       void *d_scratch, size_t scratch_bytes, float *d_tri,
                                       int64_t *d_cell, int64_t max_tri, int64_t *h_ntri,
                                       void *stream) {
    dbt_status st = check_grid(g);
    if (st != DBT_OK) return st;
    ExportBox b;
    if ((st = export_box(g, box, &b)) != DBT_OK) return st;
    if (!std::isfinite(iso)) return fail(DBT_EINVAL, "iso must be finite");
    if (!h_ntri) return fail(DBT_EINVAL, "h_ntri is NULL");
    if (max_tri < 0) return fail(DBT_EINVAL, "max_tri < 0");
    if (max_tri > 0 && !d_tri) return fail(DBT_EINVAL, "d_tri is NULL with max_tri > 0");
    if (!d_scratch || !aligned256(d_scratch)) return fail(DBT_EINVAL, "scratch must be 256-byte aligned");
    if (scratch_bytes < mc_scratch_bytes(b)) return fail(DBT_EINVAL, "scratch too small");
    const cudaStream_t s = (cudaStream_t)stream;
    const DevGrid dg = dev_grid(g);
    uint64_t lut0, lut1;
    inside_lut(g->res, iso, &lut0, &lut1);
    launch_mc_count(dg, b, lut0, lut1, d_scratch, s);
    DBT_CUDA(cudaGetLastError());
    unsigned long long total = 0;
    DBT_CUDA(cudaMemcpyAsync(&total, mc_total_ptr(d_scratch), sizeof(total), cudaMemcpyDeviceToHost, s));
    DBT_CUDA(cudaStreamSynchronize(s));
    *h_ntri = (int64_t)total;
    if (max_tri > 0 && total > 0) {
        launch_mc_emit(dg, b, g->res, iso, lut0, lut1, d_scratch, d_tri, (long long *)d_cell,
                       (long long)max_tri, s);
        DBT_CUDA(cudaGetLastError());
    }
    return DBT_OK;
}

// ------------------------------------------------------------------ quality
static bool aligned4(const void *p) { return ((uintptr_t)p & 3u) == 0; }

static dbt_status check_points(const float *p, int64_t n, const char *what) {
    if (n < 0) return fail(DBT_EINVAL, "%s: n < 0", what);
    if (n > 0 && (!p || !aligned4(p))) return fail(DBT_EINVAL, "%s: NULL or misaligned", what);
    if (n > (1ll << 31)) return fail(DBT_EINVAL, "%s: more than 2^31 points", what);
    return DBT_OK;
}

extern "C" dbt_status dbt_nn_scratch_size(int64_t n_ref, size_t *bytes) {
    if (!bytes || n_ref < 0) return fail(DBT_EINVAL, "bad argument");
    *bytes = nn_scratch_bytes(n_ref);
    return DBT_OK;
}

extern "C" dbt_status dbt_nn_distances(const float *d_ref, int64_t n_ref, const float *d_query,
                                       int64_t n_query, void *d_scratch, size_t bytes,
                                       float *d_dist, void *stream) {
    dbt_status st = check_points(d_ref, n_ref, "reference");
    if (st == DBT_OK) st = check_points(d_query, n_query, "query");
    if (st != DBT_OK) return st;
    if (n_query > 0 && !d_dist) return fail(DBT_EINVAL, "d_dist is NULL");
    if (!d_scratch || !aligned256(d_scratch) || bytes < nn_scratch_bytes(n_ref))
        return fail(DBT_EINVAL, "scratch must be 256-byte aligned and >= dbt_nn_scratch_size");
    launch_nn_distances(d_ref, n_ref, d_query, n_query, d_scratch, d_dist, (cudaStream_t)stream);
    DBT_CUDA(cudaGetLastError());
    return DBT_OK;
}

struct QualityLayout {
    size_t out, part, dpred, dgt, nn, total;
};

static QualityLayout quality_layout(int64_t n_pred, int64_t n_gt) {
    QualityLayout q;
    size_t o = 0;
    q.out = o;   o += 256;
    q.part = o;  o += up256(quality_partials_bytes());
    q.dpred = o; o += up256((size_t)n_pred * 4);
    q.dgt = o;   o += up256((size_t)n_gt * 4);
    q.nn = o;    o += nn_scratch_bytes(std::max(n_pred, n_gt));
    q.total = o;
    return q;
}

extern "C" dbt_status dbt_quality_scratch_size(int64_t n_pred, int64_t n_gt, size_t *bytes) {
    if (!bytes || n_pred < 0 || n_gt < 0) return fail(DBT_EINVAL, "bad argument");
    *bytes = quality_layout(n_pred, n_gt).total;
    return DBT_OK;
}

extern "C" dbt_status dbt_quality_metrics(const float *d_pred, int64_t n_pred, const float *d_gt,
                                          int64_t n_gt, double tolerance, void *d_scratch,
                                          size_t bytes, dbt_quality *h_out, void *stream) {
    dbt_status st = check_points(d_pred, n_pred, "predicted");
    if (st == DBT_OK) st = check_points(d_gt, n_gt, "reference");
    if (st != DBT_OK) return st;
    if (!h_out) return fail(DBT_EINVAL, "h_out is NULL");
    if (!(tolerance >= 0.0) || !std::isfinite(tolerance))
        return fail(DBT_EINVAL, "tolerance must be finite and >= 0");
    const QualityLayout q = quality_layout(n_pred, n_gt);
    if (!d_scratch || !aligned256(d_scratch) || bytes < q.total)
        return fail(DBT_EINVAL, "scratch must be 256-byte aligned and >= dbt_quality_scratch_size");
    const cudaStream_t s = (cudaStream_t)stream;
    char *base = static_cast<char *>(d_scratch);
    float *dp = reinterpret_cast<float *>(base + q.dpred);
    float *dg = reinterpret_cast<float *>(base + q.dgt);
    launch_nn_distances(d_gt, n_gt, d_pred, n_pred, base + q.nn, dp, s);    // accuracy side
    launch_nn_distances(d_pred, n_pred, d_gt, n_gt, base + q.nn, dg, s);    // completeness side
    double *out = reinterpret_cast<double *>(base + q.out);
    launch_quality_reduce(dp, n_pred, dg, n_gt, (float)tolerance, base + q.part, out, s);
    DBT_CUDA(cudaGetLastError());
    double h[6];
    DBT_CUDA(cudaMemcpyAsync(h, out, sizeof h, cudaMemcpyDeviceToHost, s));
    DBT_CUDA(cudaStreamSynchronize(s));
    h_out->accuracy = h[0];
    h_out->completeness = h[1];
    h_out->chamfer_l1 = h[2];
    h_out->precision = h[3];
    h_out->recall = h[4];
    h_out->fscore = h[5];
    h_out->n_pred = n_pred;
    h_out->n_gt = n_gt;
    return DBT_OK;
}

extern "C" dbt_status dbt_mesh_centroids(const float *d_tri, int64_t n_tri, float *d_out,
                                         void *stream) {
    dbt_status st = check_points(d_tri, n_tri, "triangles");
    if (st != DBT_OK) return st;
    if (n_tri > 0 && (!d_out || !aligned4(d_out))) return fail(DBT_EINVAL, "d_out NULL or misaligned");
    launch_centroids(d_tri, n_tri, d_out, (cudaStream_t)stream);
    DBT_CUDA(cudaGetLastError());
    return DBT_OK;
}

extern "C" dbt_status dbt_mesh_table(uint8_t *h_ntri, uint8_t *h_edges) {
    if (!h_ntri || !h_edges) return fail(DBT_EINVAL, "NULL output");
    mc_table_host(h_ntri, h_edges);
    return DBT_OK;
}

extern "C" const char *dbt_last_error(void) { return t_err; }

extern "C" const char *dbt_version(void) { return "dbtsdf 0.2.0 sm_103a"; }
