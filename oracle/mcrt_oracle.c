/*
 * mcrt_oracle.c -- FP64 analog Monte Carlo reference for the shortwave ray
 * tracer of Veerman, van Stratum & van Heerwaarden (2022), Sec. 2.3.
 *
 * TEST INFRASTRUCTURE ONLY. This file is the independent CPU oracle that the
 * CUDA path is checked against. It shares no code, header, table or constant
 * generator with the CUDA library, and the library never calls it.
 *
 * What it estimates: the same expectation as the paper's tracer (surface direct
 * and diffuse irradiance, upward flux at the domain top, 3D absorption), i.e.
 * the solution of the 3D radiative transfer equation on a periodic grid with a
 * Lambertian surface. It does so with a different, plainer algorithm:
 *
 *   - fine-cell traversal with an exact (Amanatides-Woo) DDA in double precision,
 *     free paths from the local extinction, no majorant grid (Sec. 2.3 uses a
 *     majorant grid only as an accelerator);
 *   - analog collisions: scatter with probability k_sca/k_ext, else absorbed;
 *     no photon weights and therefore no roulette (Sec. 2.3 uses weights only to
 *     speed up convergence);
 *   - analog surface: reflect with probability albedo (Lambertian), else absorbed;
 *   - two absorption estimators per cell: integer counts of analog absorptions
 *     (exact per-photon energy closure) and the track-length estimator
 *     sum(k_abs * path length), whose expectation is the same.
 *
 * Phase functions (Sec. 2.3): Rayleigh for gas, sampled by rejection;
 * Henyey-Greenstein without delta-scaling for cloud, by its inverse CDF.
 * Scatterer choice: by default cloud with probability k_sca,cloud / k_sca; the
 * paper's literal ratio k_ext,cloud / k_ext is available as mode 1.
 *
 * Random numbers: Philox4x32-10 (Salmon et al., SC'11), written here from its
 * published definition; one counter stream per photon id, so results do not
 * depend on the thread count.
 *
 * Coordinates: x east, y north, z up; grid [nz][ny][nx], x fastest; periodic in
 * x and y; surface at z = 0; domain top at z = nz*dz. The sun azimuth is
 * clockwise from north and names the direction the sun is seen in, so photons
 * travel along (-sin(sza) sin(az), -sin(sza) cos(az), -cos(sza)).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_OK 0
#define OR_EINVAL -1
#define OR_ESTEPS -2

/* ---------------- Philox4x32-10 ---------------- */

void or_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4])
{
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; ++round) {
        uint64_t a = (uint64_t)0xD2511F53u * (uint64_t)c0;
        uint64_t b = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
        uint32_t n0 = (uint32_t)(b >> 32) ^ c1 ^ k0;
        uint32_t n1 = (uint32_t)b;
        uint32_t n2 = (uint32_t)(a >> 32) ^ c3 ^ k1;
        uint32_t n3 = (uint32_t)a;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

typedef struct {
    uint32_t key[2];
    uint32_t ctr[4];
    uint32_t buf[4];
    int pos;
} stream_t;

/* Stream for one photon: counter = (id lo, id hi, block, 0x0ACE0ACE). */
static void stream_init(stream_t *s, uint64_t seed, uint64_t id)
{
    s->key[0] = (uint32_t)seed;
    s->key[1] = (uint32_t)(seed >> 32);
    s->ctr[0] = (uint32_t)id;
    s->ctr[1] = (uint32_t)(id >> 32);
    s->ctr[2] = 0;
    s->ctr[3] = 0x0ACE0ACEu;
    s->pos = 4;
}

static uint32_t stream_u32(stream_t *s)
{
    if (s->pos == 4) {
        or_philox4x32_10(s->ctr, s->key, s->buf);
        s->ctr[2] += 1;
        s->pos = 0;
    }
    return s->buf[s->pos++];
}

/* Uniform double in the open interval (0,1) from 53 random bits. */
static double stream_uniform(stream_t *s)
{
    uint64_t hi = stream_u32(s) >> 5;   /* 27 bits */
    uint64_t lo = stream_u32(s) >> 6;   /* 26 bits */
    return ((double)((hi << 26) | lo) + 0.5) * (1.0 / 9007199254740992.0);
}

/* ---------------- Sobol start positions (Sec. 2.3) ---------------- */

/* Point k of the two-dimensional Sobol sequence in natural order, as 32-bit
 * binary fractions (Sobol' 1967; Bratley & Fox 1988). Coordinate 1 is the
 * base-2 radical inverse of k: bit i-1 of k contributes 2^-i. Coordinate 2 is
 * the XOR, over the set bits i-1 of k, of the direction numbers v_i = m_i 2^-i
 * of the primitive polynomial x + 1, whose recurrence is
 * m_i = 2 m_(i-1) XOR m_(i-1) from m_1 = 1 (so m = 1, 3, 5, 15, 17, ...). */
static void sobol2_point(uint32_t k, uint32_t out[2])
{
    uint32_t x = 0, y = 0, m = 1;
    for (int i = 1; i <= 32; ++i) {
        if ((k >> (i - 1)) & 1u) {
            x ^= 1u << (32 - i);
            y ^= m << (32 - i);
        }
        m = (m << 1) ^ m;
    }
    out[0] = x;
    out[1] = y;
}

void or_sobol2(uint64_t k0, int n, uint32_t *out)
{
    for (int q = 0; q < n; ++q) sobol2_point((uint32_t)(k0 + (uint64_t)q), out + 2 * q);
}

/* ---------------- phase functions and directions (Sec. 2.3) ---------------- */

/* Rayleigh: p(mu) = 3/8 (1 + mu^2) on [-1,1]; rejection from the uniform law. */
static double sample_rayleigh(stream_t *s)
{
    for (;;) {
        double mu = 2.0 * stream_uniform(s) - 1.0;
        if (stream_uniform(s) * 2.0 <= 1.0 + mu * mu) return mu;
    }
}

/* Henyey-Greenstein by inverse CDF; g = 0 is the isotropic law. */
static double sample_hg(stream_t *s, double g)
{
    double xi = stream_uniform(s);
    if (fabs(g) < 1e-6) return 2.0 * xi - 1.0;
    double f = (1.0 - g * g) / (1.0 - g + 2.0 * g * xi);
    double mu = (1.0 + g * g - f * f) / (2.0 * g);
    if (mu > 1.0) mu = 1.0;
    if (mu < -1.0) mu = -1.0;
    return mu;
}

/* Lambertian (cosine-law) upward direction cosine. */
static double sample_lambert(stream_t *s) { return sqrt(stream_uniform(s)); }

/* New direction at angle acos(mu) from d and azimuth phi about it, built from an
 * orthonormal frame (e1, e2, d) obtained by cross products. */
static void turn(double d[3], double mu, double phi)
{
    double a[3] = {0.0, 0.0, 1.0};
    if (fabs(d[2]) > 0.9) { a[0] = 1.0; a[2] = 0.0; }
    double e1[3] = {a[1] * d[2] - a[2] * d[1], a[2] * d[0] - a[0] * d[2], a[0] * d[1] - a[1] * d[0]};
    double n1 = sqrt(e1[0] * e1[0] + e1[1] * e1[1] + e1[2] * e1[2]);
    e1[0] /= n1; e1[1] /= n1; e1[2] /= n1;
    double e2[3] = {d[1] * e1[2] - d[2] * e1[1], d[2] * e1[0] - d[0] * e1[2], d[0] * e1[1] - d[1] * e1[0]};
    double st = sqrt(fmax(0.0, 1.0 - mu * mu));
    double c = cos(phi), sn = sin(phi);
    double r[3];
    for (int q = 0; q < 3; ++q) r[q] = mu * d[q] + st * (c * e1[q] + sn * e2[q]);
    double nr = sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
    d[0] = r[0] / nr; d[1] = r[1] / nr; d[2] = r[2] / nr;
}

/* Exposed for the sampling-law tests: kind 0 Rayleigh, 1 HG(g), 2 Lambert. */
int or_sample_mu(int kind, double g, uint64_t n, uint64_t seed, double *out)
{
    stream_t s;
    stream_init(&s, seed, 0);
    for (uint64_t i = 0; i < n; ++i) {
        if (kind == 0) out[i] = sample_rayleigh(&s);
        else if (kind == 1) out[i] = sample_hg(&s, g);
        else if (kind == 2) out[i] = sample_lambert(&s);
        else return OR_EINVAL;
    }
    return OR_OK;
}

/* Exposed for the rotation tests: out[3*i..] = turn(d, mu[i], phi[i]). */
void or_turn(const double d_in[3], uint64_t n, const double *mu, const double *phi, double *out)
{
    for (uint64_t i = 0; i < n; ++i) {
        double d[3] = {d_in[0], d_in[1], d_in[2]};
        turn(d, mu[i], phi[i]);
        out[3 * i] = d[0]; out[3 * i + 1] = d[1]; out[3 * i + 2] = d[2];
    }
}

/* ---------------- scene ---------------- */

typedef struct {
    int nx, ny, nz;
    double dx, dy, dz, Lx, Ly, H;
    const float *kg, *wg, *kc, *wc, *gc, *alb;
    int pcld_mode;
} scene_t;

static void sun_direction(double sza_deg, double az_deg, double d[3])
{
    double t = sza_deg * M_PI / 180.0, p = az_deg * M_PI / 180.0;
    d[0] = -sin(t) * sin(p);
    d[1] = -sin(t) * cos(p);
    d[2] = -cos(t);
}

static inline void add_f64(double *p, double v)
{
#pragma omp atomic
    *p += v;
}

static inline void add_u64(uint64_t *p, uint64_t v)
{
#pragma omp atomic
    *p += v;
}

/* Distance along d from (x,y,z) in cell (i,j,k) to the cell's exit face;
 * *axis receives 0/1/2 for the x/y/z face that is hit first. */
static double cell_exit(const scene_t *S, const double p[3], const double d[3],
                        int i, int j, int k, int *axis)
{
    double best = INFINITY;
    int ax = 2;
    if (d[0] > 0) { double t = ((i + 1) * S->dx - p[0]) / d[0]; if (t < best) { best = t; ax = 0; } }
    else if (d[0] < 0) { double t = (i * S->dx - p[0]) / d[0]; if (t < best) { best = t; ax = 0; } }
    if (d[1] > 0) { double t = ((j + 1) * S->dy - p[1]) / d[1]; if (t < best) { best = t; ax = 1; } }
    else if (d[1] < 0) { double t = (j * S->dy - p[1]) / d[1]; if (t < best) { best = t; ax = 1; } }
    if (d[2] > 0) { double t = ((k + 1) * S->dz - p[2]) / d[2]; if (t < best) { best = t; ax = 2; } }
    else if (d[2] < 0) { double t = (k * S->dz - p[2]) / d[2]; if (t < best) { best = t; ax = 2; } }
    *axis = ax;
    return best < 0 ? 0.0 : best;
}

/* Step from cell (i,j,k) across face `axis`, placing the position exactly on
 * the face; x and y wrap periodically. */
static void cross_face(const scene_t *S, double p[3], const double d[3], int *i, int *j, int *k, int axis)
{
    if (axis == 0) {
        if (d[0] > 0) { p[0] = (*i + 1) * S->dx; if (++*i == S->nx) { *i = 0; p[0] = 0.0; } }
        else { p[0] = *i * S->dx; if (--*i < 0) { *i = S->nx - 1; p[0] = S->Lx; } }
    } else if (axis == 1) {
        if (d[1] > 0) { p[1] = (*j + 1) * S->dy; if (++*j == S->ny) { *j = 0; p[1] = 0.0; } }
        else { p[1] = *j * S->dy; if (--*j < 0) { *j = S->ny - 1; p[1] = S->Ly; } }
    } else {
        if (d[2] > 0) { p[2] = (*k + 1) * S->dz; ++*k; }
        else { p[2] = *k * S->dz; --*k; }
    }
}

typedef struct {
    double *tl_dir, *tl_dif;                     /* track-length k_abs*l per cell */
    uint64_t *n_abs_dir, *n_abs_dif;             /* analog absorptions per cell */
    uint64_t *n_sfc_dir, *n_sfc_dif, *n_sfc_abs, *n_toa;  /* per column */
    uint64_t tot[8];  /* photons, toa, atm_abs, sfc_abs, collisions, scatters, surface hits, steps */
} tally_t;

/* One analog photon history; returns 0 or OR_ESTEPS. */
static int trace_photon(const scene_t *S, const double sun[3], uint64_t seed, uint64_t id,
                        uint64_t col_offset, double diffuse_frac, int birth, uint64_t max_steps, tally_t *T,
                        uint64_t loc[8])
{
    stream_t rs;
    stream_init(&rs, seed, id);
    const uint64_t ncol = (uint64_t)S->nx * S->ny;
    uint64_t c = (id + col_offset) % ncol;
    int i = (int)(c % S->nx), j = (int)(c / S->nx), k = S->nz - 1;
    double p[3], d[3] = {sun[0], sun[1], sun[2]};
    if (birth == 1) {
        /* the k-th photon of column c takes the column's k-th Sobol point,
         * XOR-scrambled per axis by two words of its own Philox block for
         * (column, seed) (a random digital shift) */
        uint32_t pt[2], hs[4];
        uint32_t ctr[4] = {(uint32_t)c, (uint32_t)(c >> 32), 0u, 0x5C7A3B1Eu};
        uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
        sobol2_point((uint32_t)((id + col_offset) / ncol), pt);
        or_philox4x32_10(ctr, key, hs);
        p[0] = (i + ((double)(pt[0] ^ hs[0]) + 0.5) * (1.0 / 4294967296.0)) * S->dx;
        p[1] = (j + ((double)(pt[1] ^ hs[1]) + 0.5) * (1.0 / 4294967296.0)) * S->dy;
    } else {
        p[0] = (i + stream_uniform(&rs)) * S->dx;
        p[1] = (j + stream_uniform(&rs)) * S->dy;
    }
    p[2] = S->H;
    int direct = 1;
    /* Sec. 2.3: a share of the top flux enters as isotropic downwelling
     * radiance; its photons start diffuse with cosine-law downward directions */
    if (diffuse_frac > 0.0 && stream_uniform(&rs) < diffuse_frac) {
        double mu = sample_lambert(&rs);
        double phi = 2.0 * M_PI * stream_uniform(&rs);
        double st = sqrt(fmax(0.0, 1.0 - mu * mu));
        d[0] = st * cos(phi); d[1] = st * sin(phi); d[2] = -mu;
        direct = 0;
    }
    loc[0] += 1;
    uint64_t steps = 0;
    double tau = -log(stream_uniform(&rs));
    for (;;) {
        if (++steps > max_steps) { loc[7] += steps; return OR_ESTEPS; }
        size_t cell = ((size_t)k * S->ny + j) * S->nx + i;
        double kg = S->kg[cell], kc = S->kc[cell];
        double ksg = kg * S->wg[cell], ksc = kc * S->wc[cell];
        double kext = kg + kc;
        double kabs = kext - ksg - ksc;
        if (kabs < 0) kabs = 0;
        int axis;
        double s = cell_exit(S, p, d, i, j, k, &axis);
        if (kext * s >= tau) {
            /* collision inside this cell */
            double l = tau / kext;
            if (kabs > 0) add_f64(direct ? &T->tl_dir[cell] : &T->tl_dif[cell], kabs * l);
            p[0] += d[0] * l; p[1] += d[1] * l; p[2] += d[2] * l;
            loc[4] += 1;
            double u = stream_uniform(&rs);
            if (u * kext >= ksg + ksc) {            /* absorbed */
                add_u64(direct ? &T->n_abs_dir[cell] : &T->n_abs_dif[cell], 1);
                loc[2] += 1;
                break;
            }
            loc[5] += 1;
            double pc = (S->pcld_mode == 1) ? kc / kext : ksc / (ksg + ksc);
            double mu = (stream_uniform(&rs) < pc) ? sample_hg(&rs, S->gc[cell]) : sample_rayleigh(&rs);
            double phi = 2.0 * M_PI * stream_uniform(&rs);
            turn(d, mu, phi);
            direct = 0;
            tau = -log(stream_uniform(&rs));
            continue;
        }
        if (kabs > 0 && s > 0) add_f64(direct ? &T->tl_dir[cell] : &T->tl_dif[cell], kabs * s);
        tau -= kext * s;
        if (axis != 0) p[0] += d[0] * s;
        if (axis != 1) p[1] += d[1] * s;
        if (axis != 2) p[2] += d[2] * s;
        cross_face(S, p, d, &i, &j, &k, axis);
        if (k < 0) {                               /* surface */
            size_t col = (size_t)j * S->nx + i;
            add_u64(direct ? &T->n_sfc_dir[col] : &T->n_sfc_dif[col], 1);
            loc[6] += 1;
            if (stream_uniform(&rs) >= S->alb[col]) {
                add_u64(&T->n_sfc_abs[col], 1);
                loc[3] += 1;
                break;
            }
            double mu = sample_lambert(&rs);
            double phi = 2.0 * M_PI * stream_uniform(&rs);
            double st = sqrt(fmax(0.0, 1.0 - mu * mu));
            d[0] = st * cos(phi); d[1] = st * sin(phi); d[2] = mu;
            k = 0;
            p[2] = 0.0;
            direct = 0;
            tau = -log(stream_uniform(&rs));
        } else if (k >= S->nz) {                   /* leaves the domain top */
            size_t col = (size_t)j * S->nx + i;
            add_u64(&T->n_toa[col], 1);
            loc[1] += 1;
            break;
        }
    }
    loc[7] += steps;
    return OR_OK;
}

static int scene_check(const scene_t *S)
{
    if (S->nx <= 0 || S->ny <= 0 || S->nz <= 0) return OR_EINVAL;
    if (!(S->dx > 0) || !(S->dy > 0) || !(S->dz > 0)) return OR_EINVAL;
    return OR_OK;
}

/*
 * Trace photon ids [id_begin, id_end). Photon id p starts in column
 * (p + col_offset) mod (nx*ny) at a uniform position (birth 0) or at the
 * column's scrambled Sobol point number (p + col_offset) div (nx*ny) (birth 1),
 * at the domain top, along the sun beam (Sec. 2.3: rays start at the top of the domain; samples per
 * pixel = rays per column). All outputs are ACCUMULATED (+=), in raw units:
 * counts and k_abs*length [dimensionless]. totals[8] as in tally_t.tot.
 */
int or_trace(int nx, int ny, int nz, double dx, double dy, double dz,
             const float *k_gas, const float *ssa_gas, const float *k_cld,
             const float *ssa_cld, const float *g_cld, const float *albedo,
             double sza_deg, double az_deg, uint64_t id_begin, uint64_t id_end,
             uint64_t col_offset, uint64_t seed, int pcld_mode, int nthreads,
             uint64_t max_steps, double diffuse_frac, int birth,
             double *tl_dir, double *tl_dif, uint64_t *n_abs_dir, uint64_t *n_abs_dif,
             uint64_t *n_sfc_dir, uint64_t *n_sfc_dif, uint64_t *n_sfc_abs, uint64_t *n_toa,
             uint64_t *totals)
{
    scene_t S = {nx, ny, nz, dx, dy, dz, nx * dx, ny * dy, nz * dz,
                 k_gas, ssa_gas, k_cld, ssa_cld, g_cld, albedo, pcld_mode};
    if (scene_check(&S) != OR_OK || !(sza_deg >= 0.0 && sza_deg < 90.0)) return OR_EINVAL;
    if (id_end < id_begin || !(diffuse_frac >= 0.0 && diffuse_frac <= 1.0)) return OR_EINVAL;
    if (birth != 0 && birth != 1) return OR_EINVAL;
    tally_t T = {tl_dir, tl_dif, n_abs_dir, n_abs_dif, n_sfc_dir, n_sfc_dif, n_sfc_abs, n_toa, {0}};
    double sun[3];
    sun_direction(sza_deg, az_deg, sun);
    int status = OR_OK;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#endif
#pragma omp parallel
    {
        uint64_t loc[8] = {0};
        int st = OR_OK;
#pragma omp for schedule(dynamic, 1024)
        for (int64_t p = (int64_t)id_begin; p < (int64_t)id_end; ++p) {
            if (trace_photon(&S, sun, seed, (uint64_t)p, col_offset, diffuse_frac, birth, max_steps, &T, loc) !=
                OR_OK)
                st = OR_ESTEPS;
        }
#pragma omp critical
        {
            for (int q = 0; q < 8; ++q) totals[q] += loc[q];
            if (st != OR_OK) status = st;
        }
    }
    return status;
}

/*
 * Deterministic direct-beam transmittance per surface column (Sec. 2.3 defines
 * direct radiation as the never-scattered part; its expectation is Beer-Lambert
 * along the sun ray). For each column, nsub x nsub surface points on a midpoint
 * grid are traced toward the sun through the fine cells to the domain top and
 * exp(-integral of k_ext) is averaged. out[ny*nx].
 */
int or_direct_beam(int nx, int ny, int nz, double dx, double dy, double dz,
                   const float *k_gas, const float *k_cld, double sza_deg, double az_deg,
                   int nsub, int nthreads, double *out)
{
    scene_t S = {nx, ny, nz, dx, dy, dz, nx * dx, ny * dy, nz * dz,
                 k_gas, NULL, k_cld, NULL, NULL, NULL, 0};
    if (scene_check(&S) != OR_OK || nsub <= 0 || !(sza_deg >= 0.0 && sza_deg < 90.0)) return OR_EINVAL;
    double sun[3];
    sun_direction(sza_deg, az_deg, sun);
    double back[3] = {-sun[0], -sun[1], -sun[2]};     /* toward the sun */
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#endif
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t col = 0; col < (int64_t)nx * ny; ++col) {
        int ci = (int)(col % nx), cj = (int)(col / nx);
        double acc = 0.0;
        for (int a = 0; a < nsub; ++a) {
            for (int b = 0; b < nsub; ++b) {
                double p[3] = {(ci + (a + 0.5) / nsub) * dx, (cj + (b + 0.5) / nsub) * dy, 0.0};
                int i = ci, j = cj, k = 0, axis;
                double tau = 0.0;
                while (k < nz) {
                    size_t cell = ((size_t)k * ny + j) * nx + i;
                    double kext = (double)k_gas[cell] + (double)k_cld[cell];
                    double s = cell_exit(&S, p, back, i, j, k, &axis);
                    tau += kext * s;
                    if (axis != 0) p[0] += back[0] * s;
                    if (axis != 1) p[1] += back[1] * s;
                    if (axis != 2) p[2] += back[2] * s;
                    cross_face(&S, p, back, &i, &j, &k, axis);
                }
                acc += exp(-tau);
            }
        }
        out[col] = acc / ((double)nsub * nsub);
    }
    return OR_OK;
}
