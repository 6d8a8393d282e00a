/*
 * CPU oracle for in-situ multi-scattering tomography (Holodovsky et al., 2015).
 *
 * TEST INFRASTRUCTURE ONLY. This file is the plain, slow, FP64 statement of what
 * the GPU path computes. Only the tests, the smoke check and the CPU-baseline leg
 * of the benchmark load it. The product path never calls it, and it shares no
 * code, header or table with the CUDA library.
 *
 * Every function follows one passage of the paper:
 *   - optical depth / Beer-Lambert ............ Eq. tau, Eq. beer-lambert (Sec. 2)
 *   - free path by inverse transform ........... Eq. Ftau, Eq. taurand, Eq. MCextinct (Sec. 2.1.1-2.1.2)
 *   - forward MC life cycle, steps i-vi ........ Sec. 2.1.2
 *   - Henyey-Greenstein phase / sampling ....... Eq. Phg, Eq. thetaHG (squared reading, see below)
 *   - classic local estimate ................... Eq. fle (Sec. 2.1.3)
 *   - backward MC with sun local estimate ...... Eq. ble (Sec. 2.1.4)   [oracle only: reciprocity check]
 *   - voxelised scattered radiance L_c(k) ...... Eq. Lcupdate, Eq. Jc (Sec. 3.2)
 *   - LOS optical depth, transmittance ......... Eq. taoKtoc, Eq. Dvc, Eq. bTck, Eq. Tck (Sec. 3.3)
 *   - geometry matrix and image ................ Eq. IcP, Eq. PIc, Eq. Rc, Eq. IcPJbetaT, Eq. Icpixel
 *   - masked L2 cost ........................... Eq. Cost (Sec. 5.1), single channel
 *   - surrogate gradient (j fixed) ............. Eq. divCost1, Eq. Jaco1, Eq. TcofJaco1, Eq. DivTc
 *   - conditioning Q_c ......................... Sec. 6
 *   - Laplacian regulariser .................... Sec. 6 (W = identity)
 *   - full gradient: the Jacobian of Eq. DirectJacob applied to the residual, with dL/dbeta
 *     taken as the score of the free-flight density (Eq. beer-lambert, Eq. MCextinct).
 *
 * Readings where the paper is silent or garbled (each also listed in the design notes):
 *   - Eq. thetaHG is printed without the square; the inverse HG CDF used here is
 *     cos = (1 + g^2 - ((1 - g^2)/(1 - g + 2 g u))^2) / (2 g), and cos = 2u - 1 for |g| < 1e-6.
 *   - Russian roulette (step v) below rr_threshold * I0, survival probability rr_survival.
 *   - Photons enter through the top face only; every face is an open, absorbing boundary.
 *   - I0 = F cos(theta0) Lx Ly / N, so images come out in radiance units of F.
 *   - N_rays sub-pixel points are the 2-D Halton points (bases 2, 3), indices 1..N_rays.
 *   - j = 0 where beta = 0.
 *   - Random numbers: Philox-4x32-10 (Salmon et al., SC'11), key = seed, counter =
 *     (photon lo, photon hi, event, 0); u = (2 (x >> 9) + 1) / 2^24.
 *     Event 0: u0, u1 -> launch x, y; u2 -> first free path.
 *     Event s >= 1: u0 -> HG cosine, u1 -> azimuth, u2 -> roulette, u3 -> next free path.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_PI 3.14159265358979323846

/* ----------------------------------------------------------------------------------------- */
/* public structs (mirrored by the Python wrapper)                                            */

typedef struct {
    int nx, ny, nz, n_cams, n_rays, pad_;
    double h[3], o[3];
    const double *beta;      /* [nvox], x fastest, 1/m */
    const double *cam_pos;   /* [C][3] */
    const double *cam_rot;   /* [C][9]: right, up, forward */
    const int *cam_w;        /* [C] */
    const int *cam_h;        /* [C] */
    const double *cam_fov;   /* [C] horizontal field of view, rad */
    const double *reg_wz;    /* [nz] altitude weights W of the regulariser (Sec. 6), NULL: W = I */
    const double *beta_air;  /* [nvox] air (Rayleigh) extinction, or NULL; beta is then the total */
                             /* extinction beta_air + beta_aerosol (Sec. 2, two species)          */
} or_scene;

typedef struct {
    double albedo, g, sun_zenith, sun_azimuth, sun_irradiance;
    double rr_threshold, rr_survival;
    uint64_t n_photons, photon_offset, n_photons_total, seed;
    int max_order, max_events;
    double albedo_air;       /* single-scattering albedo of air (two species; ~1 in the visible) */
} or_params;

enum {
    ST_ESC0 = 0, /* 0..5: escaped weight through faces x-, x+, y-, y+, z-, z+ */
    ST_ABSORBED = 6,
    ST_RR_KILLED = 7,
    ST_RR_GAINED = 8,
    ST_FORCED = 9,
    ST_EVENTS = 10,
    ST_SEGMENTS = 11,
    ST_CAPPED = 12,
    ST_ESCAPED_N = 13,
    ST_LAUNCHED = 14,
    ST_TRACED = 15,
    ST_N = 16
};

enum { TERM_ESCAPE = 1, TERM_ABSORBED = 2, TERM_ROULETTE = 3, TERM_ORDER = 4, TERM_CAP = 5 };

/* ----------------------------------------------------------------------------------------- */
/* Philox-4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11), written from the published round     */
/* function: two 32x32->64 multiplies per round, Weyl key schedule, 10 rounds.               */

void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
        uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ k0;
        uint32_t n1 = (uint32_t)p1;
        uint32_t n2 = (uint32_t)(p0 >> 32) ^ c3 ^ k1;
        uint32_t n3 = (uint32_t)p0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

double or_u01(uint32_t x) { return (double)(2u * (x >> 9) + 1u) * (1.0 / 16777216.0); }

static void draws4(uint64_t seed, uint64_t photon, uint32_t event, uint32_t stream, double u[4]) {
    uint32_t ctr[4] = {(uint32_t)photon, (uint32_t)(photon >> 32), event, stream};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t x[4];
    or_philox4x32_10(ctr, key, x);
    for (int i = 0; i < 4; ++i) u[i] = or_u01(x[i]);
}

/* ----------------------------------------------------------------------------------------- */
/* phase function and direction sampling                                                    */

/* Eq. Phg */
double or_hg_phase(double g, double mu) {
    double d = 1.0 + g * g - 2.0 * g * mu;
    return (1.0 - g * g) / (4.0 * OR_PI * d * sqrt(d));
}

/* Eq. thetaHG, squared reading of the inverse CDF */
double or_hg_sample(double g, double u) {
    if (fabs(g) < 1e-6) return 2.0 * u - 1.0;
    double s = (1.0 - g * g) / (1.0 - g + 2.0 * g * u);
    double c = (1.0 + g * g - s * s) / (2.0 * g);
    if (c > 1.0) c = 1.0;
    if (c < -1.0) c = -1.0;
    return c;
}

/* Eq. Pray: Rayleigh phase function of air molecules */
double or_rayleigh_phase(double mu) { return 3.0 / (16.0 * OR_PI) * (1.0 + mu * mu); }

/* Eq. thetaREY: inverse CDF of Eq. Pray, cos = gamma^(1/3) - gamma^(-1/3) with
 * gamma = 4u - 2 + sqrt((4u - 2)^2 + 1) (Cardano's root of mu^3 + 3 mu + 4 - 8u = 0) */
double or_rayleigh_sample(double u) {
    const double q = 4.0 * u - 2.0;
    const double gam = q + sqrt(q * q + 1.0);
    double c = cbrt(gam) - 1.0 / cbrt(gam);
    if (c > 1.0) c = 1.0;
    if (c < -1.0) c = -1.0;
    return c;
}

/* Step iv with two species: the event's particle is air with probability beta_air / beta in
 * its voxel (Sec. 2.1.2). Its uniform comes from the bits the event's draws leave unused: each
 * of the four uniforms of or_u01 takes the top 23 bits of its word, so the low 9 bits of words
 * 0 and 1 and the low 5 bits of word 2 form a 23-bit integer m, independent of the other four
 * draws, and u = (2m + 1) / 2^24 like or_u01. */
double or_particle_uniform(uint64_t seed, uint64_t photon, uint32_t event) {
    uint32_t ctr[4] = {(uint32_t)photon, (uint32_t)(photon >> 32), event, 0u};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t x[4];
    or_philox4x32_10(ctr, key, x);
    const uint32_t m = (x[0] & 511u) | ((x[1] & 511u) << 9) | ((x[2] & 31u) << 18);
    return (2.0 * (double)m + 1.0) * (1.0 / 16777216.0);
}

/* New direction at polar cosine ct and azimuth phi about d. The transverse frame is
 * e2 = normalize(a x d), e1 = e2 x d with reference axis a = z, or a = x when |d_z| >= 0.9. */
void or_rotate(const double d[3], double ct, double phi, double out[3]) {
    double st = sqrt(fmax(0.0, 1.0 - ct * ct));
    double cp = cos(phi), sp = sin(phi);
    double e1[3], e2[3];
    if (fabs(d[2]) < 0.9) {
        double n = sqrt(d[0] * d[0] + d[1] * d[1]);
        e2[0] = -d[1] / n; e2[1] = d[0] / n; e2[2] = 0.0;
    } else {
        double n = sqrt(d[1] * d[1] + d[2] * d[2]);
        e2[0] = 0.0; e2[1] = -d[2] / n; e2[2] = d[1] / n;
    }
    e1[0] = e2[1] * d[2] - e2[2] * d[1];
    e1[1] = e2[2] * d[0] - e2[0] * d[2];
    e1[2] = e2[0] * d[1] - e2[1] * d[0];
    for (int a = 0; a < 3; ++a) out[a] = st * (cp * e1[a] + sp * e2[a]) + ct * d[a];
}

/* ----------------------------------------------------------------------------------------- */
/* grid geometry and voxel traversal (Amanatides-Woo)                                        */

static inline int dim(const or_scene *s, int a) { return a == 0 ? s->nx : (a == 1 ? s->ny : s->nz); }
static inline long nvox_of(const or_scene *s) { return (long)s->nx * s->ny * s->nz; }
static inline long lin(const or_scene *s, const int v[3]) { return v[0] + (long)s->nx * (v[1] + (long)s->ny * v[2]); }

static int coord_vox(const or_scene *s, int a, double x) {
    double f = floor((x - s->o[a]) / s->h[a]);
    int n = dim(s, a);
    if (f < 0) return 0;
    if (f > n - 1) return n - 1;
    return (int)f;
}

typedef struct {
    double O[3], d[3], tmax[3], tdel[3], t;
    int ix[3], step[3];
} or_ray;

static void ray_init(const or_scene *s, or_ray *r, const double O[3], const double d[3], const int v[3], double t0) {
    for (int a = 0; a < 3; ++a) {
        r->O[a] = O[a];
        r->d[a] = d[a];
        r->ix[a] = v[a];
        double lo = s->o[a] + v[a] * s->h[a];
        if (d[a] > 0) {
            r->step[a] = 1;
            r->tmax[a] = (lo + s->h[a] - O[a]) / d[a];
            r->tdel[a] = s->h[a] / d[a];
        } else if (d[a] < 0) {
            r->step[a] = -1;
            r->tmax[a] = (lo - O[a]) / d[a];
            r->tdel[a] = -s->h[a] / d[a];
        } else {
            r->step[a] = 0;
            r->tmax[a] = INFINITY;
            r->tdel[a] = INFINITY;
        }
    }
    r->t = t0;
}

/* axis of the next face crossing; ties go to x, then y, then z */
static inline int ray_axis(const or_ray *r) {
    int a = 0;
    if (r->tmax[1] < r->tmax[a]) a = 1;
    if (r->tmax[2] < r->tmax[a]) a = 2;
    return a;
}

/* crosses the face on axis a; returns 1 when the ray has left the grid */
static inline int ray_step(const or_scene *s, or_ray *r, int a) {
    r->t = r->tmax[a];
    r->ix[a] += r->step[a];
    r->tmax[a] += r->tdel[a];
    return r->ix[a] < 0 || r->ix[a] >= dim(s, a);
}

typedef void (*visit_fn)(void *ctx, long k, double len);

/* Sums over the voxels a ray crosses from parameter t0 to t_end (or to the grid exit).
 * Returns the exit face (0..5) if the ray left the grid before t_end, else -1. */
static int walk(const or_scene *s, const double O[3], const double d[3], const int v[3], double t0, double t_end,
                visit_fn fn, void *ctx) {
    or_ray r;
    ray_init(s, &r, O, d, v, t0);
    for (;;) {
        int a = ray_axis(&r);
        double te = r.tmax[a] < t_end ? r.tmax[a] : t_end;
        double len = te - r.t;
        if (len < 0) len = 0;
        fn(ctx, lin(s, r.ix), len);
        if (r.tmax[a] >= t_end) return -1;
        if (ray_step(s, &r, a)) return 2 * a + (r.step[a] > 0);
    }
}

/* Clips a ray from X along d to the grid box. Returns 0 if it misses. */
static int ray_enter(const or_scene *s, const double X[3], const double d[3], int v[3], double *t0) {
    double tn = 0.0, tf = INFINITY;
    for (int a = 0; a < 3; ++a) {
        double lo = s->o[a], hi = s->o[a] + dim(s, a) * s->h[a];
        if (d[a] == 0.0) {
            if (X[a] < lo || X[a] > hi) return 0;
        } else {
            double t1 = (lo - X[a]) / d[a], t2 = (hi - X[a]) / d[a];
            if (t1 > t2) { double tt = t1; t1 = t2; t2 = tt; }
            if (t1 > tn) tn = t1;
            if (t2 < tf) tf = t2;
        }
    }
    if (!(tn < tf)) return 0;
    for (int a = 0; a < 3; ++a) v[a] = coord_vox(s, a, X[a] + tn * d[a]);
    *t0 = tn;
    return 1;
}

/* ----------------------------------------------------------------------------------------- */
/* camera model: pinhole, d = normalize(f + x r + y u)                                       */

static long pix_offset(const or_scene *s, int c) {
    long off = 0;
    for (int i = 0; i < c; ++i) off += (long)s->cam_w[i] * s->cam_h[i];
    return off;
}
static long total_pixels(const or_scene *s) { return pix_offset(s, s->n_cams); }

static void cam_tan(const or_scene *s, int c, double *tx, double *ty) {
    *tx = tan(0.5 * s->cam_fov[c]);
    *ty = *tx * (double)s->cam_h[c] / (double)s->cam_w[c];
}

/* direction through image-plane point (px, py), px in [0, W], py in [0, H] */
static void pixel_dir(const or_scene *s, int c, double px, double py, double d[3]) {
    double tx, ty;
    cam_tan(s, c, &tx, &ty);
    double x = (2.0 * px / s->cam_w[c] - 1.0) * tx;
    double y = (2.0 * py / s->cam_h[c] - 1.0) * ty;
    const double *R = s->cam_rot + 9 * c;
    double n2 = 0;
    for (int a = 0; a < 3; ++a) {
        d[a] = R[6 + a] + x * R[a] + y * R[3 + a];
        n2 += d[a] * d[a];
    }
    double n = sqrt(n2);
    for (int a = 0; a < 3; ++a) d[a] /= n;
}

double or_radical_inverse(int base, int i) {
    double f = 1.0, r = 0.0;
    while (i > 0) {
        f /= base;
        r += f * (i % base);
        i /= base;
    }
    return r;
}

/* exact solid angle of the image-plane rectangle [x1,x2]x[y1,y2] at unit focal distance */
static double rect_solid_angle(double x1, double x2, double y1, double y2) {
#define FSA(x, y) atan((x) * (y) / sqrt(1.0 + (x) * (x) + (y) * (y)))
    return FSA(x2, y2) - FSA(x1, y2) - FSA(x2, y1) + FSA(x1, y1);
#undef FSA
}

/* pixel index of the point X seen by camera c, or -1 */
static long project(const or_scene *s, int c, const double X[3], double *omega) {
    const double *R = s->cam_rot + 9 * c, *P = s->cam_pos + 3 * c;
    double v[3] = {X[0] - P[0], X[1] - P[1], X[2] - P[2]};
    double zc = v[0] * R[6] + v[1] * R[7] + v[2] * R[8];
    if (!(zc > 0)) return -1;
    double x = (v[0] * R[0] + v[1] * R[1] + v[2] * R[2]) / zc;
    double y = (v[0] * R[3] + v[1] * R[4] + v[2] * R[5]) / zc;
    double tx, ty;
    cam_tan(s, c, &tx, &ty);
    int W = s->cam_w[c], H = s->cam_h[c];
    double px = (x / tx + 1.0) * 0.5 * W, py = (y / ty + 1.0) * 0.5 * H;
    double fi = floor(px), fj = floor(py);
    if (fi < 0 || fj < 0 || fi >= W || fj >= H) return -1;
    int i = (int)fi, j = (int)fj;
    double x1 = (2.0 * i / W - 1.0) * tx, x2 = (2.0 * (i + 1) / W - 1.0) * tx;
    double y1 = (2.0 * j / H - 1.0) * ty, y2 = (2.0 * (j + 1) / H - 1.0) * ty;
    *omega = rect_solid_angle(x1, x2, y1, y2);
    return (long)j * W + i;
}

/* ----------------------------------------------------------------------------------------- */
/* optical depth along a segment (Eq. tau) with the visit callback                            */

typedef struct { const double *beta; double tau; } tau_ctx;
static void tau_visit(void *c, long k, double len) {
    tau_ctx *t = (tau_ctx *)c;
    t->tau += t->beta[k] * len;
}

/* adds weight * (length in voxel m) to g[m] along the segment from X (in voxel v) to point Y */
typedef struct { double *g; double weight; } scatter_ctx;
static void scatter_visit(void *c, long k, double len) {
    scatter_ctx *t = (scatter_ctx *)c;
    t->g[k] += t->weight * len;
}

static void shadow_scatter(const or_scene *s, const double X[3], const int v[3], const double Y[3], double weight,
                           double *g) {
    double d[3] = {Y[0] - X[0], Y[1] - X[1], Y[2] - X[2]};
    double dist = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    if (dist == 0.0) return;
    for (int a = 0; a < 3; ++a) d[a] /= dist;
    scatter_ctx t = {g, weight};
    walk(s, X, d, v, 0.0, dist, scatter_visit, &t);
}

/* optical depth from X (in voxel v) to point Y, clipped to the grid */
static double tau_to_point(const or_scene *s, const double X[3], const int v[3], const double Y[3]) {
    double d[3] = {Y[0] - X[0], Y[1] - X[1], Y[2] - X[2]};
    double dist = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    if (dist == 0.0) return 0.0;
    for (int a = 0; a < 3; ++a) d[a] /= dist;
    tau_ctx t = {s->beta, 0.0};
    walk(s, X, d, v, 0.0, dist, tau_visit, &t);
    return t.tau;
}

/* ----------------------------------------------------------------------------------------- */
/* forward MC photon transport (Sec. 2.1.2) with voxelised (Eq. Lcupdate) and classic        */
/* (Eq. fle) local estimates, and path recording for the full gradient                       */

typedef struct {
    /* path record of one photon (full gradient) */
    long *seg_k;
    double *seg_len;
    int *flight_of_seg;
    long n_seg, cap_seg;
    long *ev_k;     /* event voxel, 1-based event index s -> ev_k[s-1] */
    double *ev_w;   /* w_s = sum_c a_c(k_s) * albedo * I_s * P_c(s) */
    int *ev_air;    /* event s scattered off air (two species) */
    long n_ev, cap_ev;
} path_rec;

typedef struct {
    const or_scene *s;
    const or_params *P;
    double sun[3], I0, ext[3];
    long nvox;
    double *L;         /* [C][nvox] or NULL */
    double *cimg;      /* classic images [sum W*H] or NULL */
    double *stats;     /* [ST_N] */
    const double *adj; /* a_c(k) [C][nvox] or NULL (full gradient replay) */
    const double *cres; /* dE/di per pixel [sum W*H] or NULL (classic-estimator gradient replay) */
    double *gsh;       /* [nvox] receives the shadow-ray terms of the classic-estimator gradient */
    path_rec *rec;     /* non-NULL in full-gradient replay */
    double last[3];    /* the traced photon's last event point (its launch point before any) */
} tctx;

static void rec_seg(path_rec *r, long k, double len, int flight) {
    if (!r) return;
    if (r->n_seg == r->cap_seg) {
        r->cap_seg = r->cap_seg ? 2 * r->cap_seg : 256;
        r->seg_k = (long *)realloc(r->seg_k, r->cap_seg * sizeof(long));
        r->seg_len = (double *)realloc(r->seg_len, r->cap_seg * sizeof(double));
        r->flight_of_seg = (int *)realloc(r->flight_of_seg, r->cap_seg * sizeof(int));
    }
    r->seg_k[r->n_seg] = k;
    r->seg_len[r->n_seg] = len;
    r->flight_of_seg[r->n_seg] = flight;
    r->n_seg++;
}

static void rec_event(path_rec *r, long k, double w, int air) {
    if (!r) return;
    if (r->n_ev == r->cap_ev) {
        r->cap_ev = r->cap_ev ? 2 * r->cap_ev : 64;
        r->ev_k = (long *)realloc(r->ev_k, r->cap_ev * sizeof(long));
        r->ev_w = (double *)realloc(r->ev_w, r->cap_ev * sizeof(double));
        r->ev_air = (int *)realloc(r->ev_air, r->cap_ev * sizeof(int));
    }
    r->ev_k[r->n_ev] = k;
    r->ev_w[r->n_ev] = w;
    r->ev_air[r->n_ev] = air;
    r->n_ev++;
}

/* Step ii-iii: free flight of optical depth tau from X (in voxel v) along d.
 * Returns 1 on collision (Xn, vn set), 0 on escape (*face set). */
static int flight(tctx *c, const double X[3], const double d[3], const int v[3], double tau, double Xn[3], int vn[3],
                  int *face, int flight_no) {
    const or_scene *s = c->s;
    or_ray r;
    ray_init(s, &r, X, d, v, 0.0);
    for (;;) {
        long k = lin(s, r.ix);
        c->stats[ST_SEGMENTS] += 1.0;
        int a = ray_axis(&r);
        double seg = r.tmax[a] - r.t;
        if (seg < 0) seg = 0;
        double b = s->beta[k];
        if (tau <= b * seg) {
            double l = tau / b;
            for (int q = 0; q < 3; ++q) Xn[q] = X[q] + (r.t + l) * d[q];
            vn[0] = r.ix[0]; vn[1] = r.ix[1]; vn[2] = r.ix[2];
            rec_seg(c->rec, k, l, flight_no);
            return 1;
        }
        tau -= b * seg;
        rec_seg(c->rec, k, seg, flight_no);
        if (ray_step(s, &r, a)) {
            *face = 2 * a + (r.step[a] > 0);
            return 0;
        }
    }
}

#define FNV_OFFSET 2166136261u
#define FNV_PRIME 16777619u

/* One photon packet, steps i-vi. Returns the path checksum. */
static uint32_t trace_photon(tctx *c, uint64_t p) {
    const or_scene *s = c->s;
    const or_params *P = c->P;
    double u[4];
    draws4(P->seed, p, 0, 0, u);
    /* step i: launch uniformly over the top face along the sun direction */
    double X[3] = {s->o[0] + u[0] * c->ext[0], s->o[1] + u[1] * c->ext[1], s->o[2] + c->ext[2]};
    int v[3] = {coord_vox(s, 0, X[0]), coord_vox(s, 1, X[1]), s->nz - 1};
    double d[3] = {c->sun[0], c->sun[1], c->sun[2]};
    double I = c->I0;
    double tau = -log(1.0 - u[2]);
    for (int q = 0; q < 3; ++q) c->last[q] = X[q];
    c->stats[ST_LAUNCHED] += I;
    c->stats[ST_TRACED] += 1.0;
    uint32_t hash = FNV_OFFSET;
    uint32_t s_ev = 0;
    int term;
    for (;;) {
        double Xn[3];
        int vn[3], face = -1;
        if (!flight(c, X, d, v, tau, Xn, vn, &face, (int)s_ev + 1)) {
            c->stats[ST_ESC0 + face] += I;
            c->stats[ST_ESCAPED_N] += 1.0;
            term = TERM_ESCAPE;
            break;
        }
        s_ev += 1;
        for (int q = 0; q < 3; ++q) c->last[q] = Xn[q];
        long k = lin(s, vn);
        hash = (hash ^ (uint32_t)k) * FNV_PRIME;
        c->stats[ST_EVENTS] += 1.0;
        /* step iv: the particle (one species unless the scene has air) and its albedo */
        int air = 0;
        if (s->beta_air) air = or_particle_uniform(P->seed, p, s_ev) * s->beta[k] < s->beta_air[k];
        const double alb = air ? P->albedo_air : P->albedo;
        /* local estimates toward every camera (Eq. Lcupdate; Eq. fle) */
        double w = 0.0;
        for (int cam = 0; cam < s->n_cams; ++cam) {
            const double *Pc = s->cam_pos + 3 * cam;
            double vv[3] = {Pc[0] - Xn[0], Pc[1] - Xn[1], Pc[2] - Xn[2]};
            double r2 = vv[0] * vv[0] + vv[1] * vv[1] + vv[2] * vv[2];
            if (r2 == 0.0) continue;
            double rr = sqrt(r2);
            double mu = (d[0] * vv[0] + d[1] * vv[1] + d[2] * vv[2]) / rr;
            double contrib = alb * I * (air ? or_rayleigh_phase(mu) : or_hg_phase(P->g, mu));
            if (c->L) c->L[(long)cam * c->nvox + k] += contrib;
            if (c->adj) w += c->adj[(long)cam * c->nvox + k] * contrib;
            if (c->cimg) {
                double omega;
                long pix = project(s, cam, Xn, &omega);
                if (pix >= 0) {
                    double t = exp(-tau_to_point(s, Xn, vn, Pc));
                    c->cimg[pix_offset(s, cam) + pix] += contrib * t / (r2 * omega);
                }
            }
            if (c->cres) {  /* classic-estimator gradient: f_s weighted by its pixel's dE/di */
                double omega;
                long pix = project(s, cam, Xn, &omega);
                if (pix >= 0) {
                    const double cr = c->cres[pix_offset(s, cam) + pix];
                    if (cr != 0.0) {
                        const double f = contrib * exp(-tau_to_point(s, Xn, vn, Pc)) / (r2 * omega);
                        w += cr * f;
                        /* d f / d beta_m = -f * (length of the shadow ray in voxel m) */
                        shadow_scatter(s, Xn, vn, Pc, -cr * f, c->gsh);
                    }
                }
            }
        }
        rec_event(c->rec, k, w, air);
        /* step v: albedo weighting and Russian roulette */
        c->stats[ST_ABSORBED] += (1.0 - alb) * I;
        I *= alb;
        if (I == 0.0) { term = TERM_ABSORBED; break; }
        if (P->max_order > 0 && (int)s_ev >= P->max_order) {
            c->stats[ST_FORCED] += I;
            term = TERM_ORDER;
            break;
        }
        if ((int)s_ev >= P->max_events) {
            c->stats[ST_FORCED] += I;
            c->stats[ST_CAPPED] += 1.0;
            term = TERM_CAP;
            break;
        }
        draws4(P->seed, p, s_ev, 0, u);
        if (I < P->rr_threshold * c->I0) {
            if (u[2] < P->rr_survival) {
                c->stats[ST_RR_GAINED] += I * (1.0 / P->rr_survival - 1.0);
                I /= P->rr_survival;
            } else {
                c->stats[ST_RR_KILLED] += I;
                term = TERM_ROULETTE;
                break;
            }
        }
        /* step vi: new direction by the particle's inverse transform, uniform azimuth */
        double ct = air ? or_rayleigh_sample(u[0]) : or_hg_sample(P->g, u[0]);
        double nd[3];
        or_rotate(d, ct, 2.0 * OR_PI * u[1], nd);
        for (int q = 0; q < 3; ++q) { X[q] = Xn[q]; d[q] = nd[q]; v[q] = vn[q]; }
        tau = -log(1.0 - u[3]);
    }
    hash = (hash ^ s_ev) * FNV_PRIME;
    hash = (hash ^ (uint32_t)term) * FNV_PRIME;
    return hash;
}

static void tctx_init(tctx *c, const or_scene *s, const or_params *P) {
    memset(c, 0, sizeof(*c));
    c->s = s;
    c->P = P;
    double th = P->sun_zenith, ph = P->sun_azimuth;
    c->sun[0] = -sin(th) * cos(ph);
    c->sun[1] = -sin(th) * sin(ph);
    c->sun[2] = -cos(th);
    c->ext[0] = s->nx * s->h[0];
    c->ext[1] = s->ny * s->h[1];
    c->ext[2] = s->nz * s->h[2];
    double N = (double)(P->n_photons_total ? P->n_photons_total : P->n_photons);
    c->I0 = P->sun_irradiance * cos(th) * c->ext[0] * c->ext[1] / N;
    c->nvox = nvox_of(s);
}

/* The deterministic stages run on the OpenMP default team; a call that asks for a thread count
 * sets it for its whole duration (and restores it), so that every stage uses that many. */
static int threads_begin(int req) {
#ifdef _OPENMP
    const int prev = omp_get_max_threads();
    if (req > 0) omp_set_num_threads(req);
    return prev;
#else
    (void)req;
    return 1;
#endif
}

static void threads_end(int prev) {
#ifdef _OPENMP
    omp_set_num_threads(prev);
#else
    (void)prev;
#endif
}

static int nthreads_of(int req) {
#ifdef _OPENMP
    return req > 0 ? req : omp_get_max_threads();
#else
    (void)req;
    return 1;
#endif
}

/* Forward render: L [C][nvox] (may be NULL), classic images (may be NULL), stats [16],
 * per-photon hash (may be NULL), skip mask (may be NULL: photons with skip[p] != 0 are
 * not traced), per-photon last event point [n][3] in grid coordinates (may be NULL; the launch
 * point for a photon without events). Photon ids run from photon_offset to
 * photon_offset + n_photons - 1. */
void or_render(const or_scene *s, const or_params *P, double *L, double *cimg, double *stats, uint32_t *hash,
               const uint8_t *skip, int nthreads, double *last_pt) {
    const long nvox = nvox_of(s);
    const long nL = (long)s->n_cams * nvox, nI = total_pixels(s);
    int nt = nthreads_of(nthreads);
    double *accL = L ? (double *)calloc((size_t)nt * nL, sizeof(double)) : NULL;
    double *accI = cimg ? (double *)calloc((size_t)nt * nI, sizeof(double)) : NULL;
    double *accS = (double *)calloc((size_t)nt * ST_N, sizeof(double));
    const long n = (long)P->n_photons;
#pragma omp parallel num_threads(nt)
    {
        int tid = 0;
#ifdef _OPENMP
        tid = omp_get_thread_num();
#endif
        tctx c;
        tctx_init(&c, s, P);
        c.L = accL ? accL + (size_t)tid * nL : NULL;
        c.cimg = accI ? accI + (size_t)tid * nI : NULL;
        c.stats = accS + (size_t)tid * ST_N;
#pragma omp for schedule(static, 4096)
        for (long i = 0; i < n; ++i) {
            if (skip && skip[i]) {
                if (hash) hash[i] = 0;
                continue;
            }
            uint32_t h = trace_photon(&c, P->photon_offset + (uint64_t)i);
            if (hash) hash[i] = h;
            if (last_pt)
                for (int q = 0; q < 3; ++q) last_pt[3 * i + q] = c.last[q] - s->o[q];
        }
    }
    for (int t = 0; t < nt; ++t) {
        if (L) for (long i = 0; i < nL; ++i) L[i] = (t ? L[i] : 0.0) + accL[(size_t)t * nL + i];
        if (cimg) for (long i = 0; i < nI; ++i) cimg[i] = (t ? cimg[i] : 0.0) + accI[(size_t)t * nI + i];
        for (int i = 0; i < ST_N; ++i) stats[i] = (t ? stats[i] : 0.0) + accS[(size_t)t * ST_N + i];
    }
    free(accL);
    free(accI);
    free(accS);
}

/* ----------------------------------------------------------------------------------------- */
/* LOS transmittance (Eq. taoKtoc, Eq. Tck): from the centre of voxel k to X_c               */

void or_transmittance(const or_scene *s, double *tau_out, double *T_out) {
    const long nvox = nvox_of(s);
    for (int c = 0; c < s->n_cams; ++c) {
        const double *Pc = s->cam_pos + 3 * c;
#pragma omp parallel for schedule(static)
        for (long k = 0; k < nvox; ++k) {
            int v[3] = {(int)(k % s->nx), (int)((k / s->nx) % s->ny), (int)(k / ((long)s->nx * s->ny))};
            double X[3];
            for (int a = 0; a < 3; ++a) X[a] = s->o[a] + (v[a] + 0.5) * s->h[a];
            double tau = tau_to_point(s, X, v, Pc);
            if (tau_out) tau_out[(long)c * nvox + k] = tau;
            if (T_out) T_out[(long)c * nvox + k] = exp(-tau);
        }
    }
}

/* W_c^T s (Eq. Dvc transposed): gT[c][m] = sum_k W_c(k, m) s[c][k] */
typedef struct { double *g; double w; } scat_ctx;
static void scat_visit(void *cc, long k, double len) {
    scat_ctx *c = (scat_ctx *)cc;
    c->g[k] += c->w * len;
}

void or_los_adjoint(const or_scene *s, const double *sv, double *gT) {
    const long nvox = nvox_of(s);
    memset(gT, 0, sizeof(double) * (size_t)s->n_cams * nvox);
    /* one camera per thread: each camera's rows are summed by one thread in voxel order, so the
     * result does not depend on the thread count */
#pragma omp parallel for schedule(dynamic, 1)
    for (int c = 0; c < s->n_cams; ++c) {
        const double *Pc = s->cam_pos + 3 * c;
        for (long k = 0; k < nvox; ++k) {
            double w = sv[(long)c * nvox + k];
            if (w == 0.0) continue;
            int v[3] = {(int)(k % s->nx), (int)((k / s->nx) % s->ny), (int)(k / ((long)s->nx * s->ny))};
            double X[3], d[3];
            for (int a = 0; a < 3; ++a) X[a] = s->o[a] + (v[a] + 0.5) * s->h[a];
            for (int a = 0; a < 3; ++a) d[a] = Pc[a] - X[a];
            double dist = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
            if (dist == 0.0) continue;
            for (int a = 0; a < 3; ++a) d[a] /= dist;
            scat_ctx sc = {gT + (long)c * nvox, w};
            walk(s, X, d, v, 0.0, dist, scat_visit, &sc);
        }
    }
}

/* ----------------------------------------------------------------------------------------- */
/* pixel rays: image formation (Eq. Icpixel), back-projection (Pi^T), ray counts (Q_c)      */

typedef struct { const double *L, *T; double acc; } img_ctx;
static void img_visit(void *cc, long k, double len) {
    img_ctx *c = (img_ctx *)cc;
    c->acc += len * c->L[k] * c->T[k];
}

/* i_c(p) = 1/(N_rays V) sum_rho sum_k l(k) L_c(k) T_c(k) */
void or_images(const or_scene *s, const double *L, const double *T, double *img) {
    const long nvox = nvox_of(s);
    const double V = s->h[0] * s->h[1] * s->h[2];
    for (int c = 0; c < s->n_cams; ++c) {
        const int W = s->cam_w[c], H = s->cam_h[c];
        const long off = pix_offset(s, c);
        const double *Pc = s->cam_pos + 3 * c;
#pragma omp parallel for schedule(static)
        for (long p = 0; p < (long)W * H; ++p) {
            int i = (int)(p % W), j = (int)(p / W);
            img_ctx ic = {L + (long)c * nvox, T + (long)c * nvox, 0.0};
            for (int rho = 1; rho <= s->n_rays; ++rho) {
                double d[3], t0;
                int v[3];
                pixel_dir(s, c, i + or_radical_inverse(2, rho), j + or_radical_inverse(3, rho), d);
                if (!ray_enter(s, Pc, d, v, &t0)) continue;
                walk(s, Pc, d, v, t0, INFINITY, img_visit, &ic);
            }
            img[off + p] = ic.acc / (s->n_rays * V);
        }
    }
}

/* b_c(k) = sum_p Pi_c(p, k) rr(p) */
void or_backproject(const or_scene *s, const double *rr, double *b) {
    const long nvox = nvox_of(s);
    const double V = s->h[0] * s->h[1] * s->h[2];
    memset(b, 0, sizeof(double) * (size_t)s->n_cams * nvox);
    /* one camera per thread, its pixels in order: independent of the thread count */
#pragma omp parallel for schedule(dynamic, 1)
    for (int c = 0; c < s->n_cams; ++c) {
        const int W = s->cam_w[c], H = s->cam_h[c];
        const long off = pix_offset(s, c);
        const double *Pc = s->cam_pos + 3 * c;
        for (long p = 0; p < (long)W * H; ++p) {
            double w = rr[off + p];
            if (w == 0.0) continue;
            int i = (int)(p % W), j = (int)(p / W);
            for (int rho = 1; rho <= s->n_rays; ++rho) {
                double d[3], t0;
                int v[3];
                pixel_dir(s, c, i + or_radical_inverse(2, rho), j + or_radical_inverse(3, rho), d);
                if (!ray_enter(s, Pc, d, v, &t0)) continue;
                scat_ctx sc = {b + (long)c * nvox, w / (s->n_rays * V)};
                walk(s, Pc, d, v, t0, INFINITY, scat_visit, &sc);
            }
        }
    }
}

typedef struct { double *q; double eps; } cnt_ctx;
static void cnt_visit(void *cc, long k, double len) {
    cnt_ctx *c = (cnt_ctx *)cc;
    if (len >= c->eps) c->q[k] += 1.0;
}

/* Q_c(k): number of sub-pixel rays through voxel k (Sec. 6). A ray counts when its chord in
 * the voxel is at least 1e-4 of the smallest voxel edge, so rays that only graze an edge or a
 * corner (chord ~ 0) are not counted. */
void or_ray_counts(const or_scene *s, double *Q) {
    const long nvox = nvox_of(s);
    memset(Q, 0, sizeof(double) * (size_t)s->n_cams * nvox);
    for (int c = 0; c < s->n_cams; ++c) {
        const int W = s->cam_w[c], H = s->cam_h[c];
        const double *Pc = s->cam_pos + 3 * c;
        double hmin = s->h[0] < s->h[1] ? s->h[0] : s->h[1];
        if (s->h[2] < hmin) hmin = s->h[2];
        cnt_ctx cc = {Q + (long)c * nvox, 1e-4 * hmin};
        for (long p = 0; p < (long)W * H; ++p) {
            int i = (int)(p % W), j = (int)(p / W);
            for (int rho = 1; rho <= s->n_rays; ++rho) {
                double d[3], t0;
                int v[3];
                pixel_dir(s, c, i + or_radical_inverse(2, rho), j + or_radical_inverse(3, rho), d);
                if (!ray_enter(s, Pc, d, v, &t0)) continue;
                walk(s, Pc, d, v, t0, INFINITY, cnt_visit, &cc);
            }
        }
    }
}

/* ----------------------------------------------------------------------------------------- */
/* sun mask M_c of Eq. Cost: 0 for the pixels whose centre ray lies within radius of the      */
/* direction to the sun, 1 elsewhere                                                         */

void or_sun_mask(const or_scene *s, double zenith, double azimuth, double radius, uint8_t *mask) {
    const double to_sun[3] = {sin(zenith) * cos(azimuth), sin(zenith) * sin(azimuth), cos(zenith)};
    long off = 0;
    for (int c = 0; c < s->n_cams; ++c) {
        const int w = s->cam_w[c], h = s->cam_h[c];
        for (int j = 0; j < h; ++j)
            for (int i = 0; i < w; ++i) {
                double d[3];
                pixel_dir(s, c, i + 0.5, j + 0.5, d);
                const double cosang = d[0] * to_sun[0] + d[1] * to_sun[1] + d[2] * to_sun[2];
                const double ang = acos(cosang > 1.0 ? 1.0 : (cosang < -1.0 ? -1.0 : cosang));
                mask[off + (long)j * w + i] = ang < radius ? 0 : 1;
            }
        off += (long)w * h;
    }
}

/* ----------------------------------------------------------------------------------------- */
/* regulariser: Psi = || W Lap beta ||^2 with the 6-neighbour graph Laplacian and W diagonal */
/* in altitude (the scene's reg_wz per layer; identity when it is NULL)                      */

void or_laplacian(const or_scene *s, const double *beta, double *psi, double *grad) {
    /* Psi = |W Lap beta|^2 with the 6-neighbour graph Laplacian and W diagonal, W_kk = the    */
    /* altitude weight of voxel k's layer (Sec. 6); dPsi = 2 Lap^T W^T W Lap beta.             */
    const long nvox = nvox_of(s);
    double *lb = (double *)calloc((size_t)nvox, sizeof(double));
    const int n[3] = {s->nx, s->ny, s->nz};
    for (long k = 0; k < nvox; ++k) {
        int v[3] = {(int)(k % s->nx), (int)((k / s->nx) % s->ny), (int)(k / ((long)s->nx * s->ny))};
        double acc = 0.0;
        for (int a = 0; a < 3; ++a)
            for (int sg = -1; sg <= 1; sg += 2) {
                int w[3] = {v[0], v[1], v[2]};
                w[a] += sg;
                if (w[a] < 0 || w[a] >= n[a]) continue;
                acc += beta[lin(s, w)] - beta[k];
            }
        lb[k] = acc;                      /* (Lap beta)_k */
    }
    double ps = 0.0;
    for (long k = 0; k < nvox; ++k) {
        const double wk = s->reg_wz ? s->reg_wz[k / ((long)s->nx * s->ny)] : 1.0;
        ps += (wk * lb[k]) * (wk * lb[k]);
        lb[k] *= wk * wk;                 /* now (W^T W Lap beta)_k */
    }
    *psi = ps;
    if (grad) {
        /* the graph Laplacian is symmetric: Lap^T = Lap */
        for (long k = 0; k < nvox; ++k) {
            int v[3] = {(int)(k % s->nx), (int)((k / s->nx) % s->ny), (int)(k / ((long)s->nx * s->ny))};
            double acc = 0.0;
            for (int a = 0; a < 3; ++a)
                for (int sg = -1; sg <= 1; sg += 2) {
                    int w[3] = {v[0], v[1], v[2]};
                    w[a] += sg;
                    if (w[a] < 0 || w[a] >= n[a]) continue;
                    acc += lb[lin(s, w)] - lb[k];
                }
            grad[k] = 2.0 * acc;
        }
    }
    free(lb);
}

/* the regulariser acts on the variable field: beta_aerosol = beta - beta_air */
static void laplacian_of_aerosol(const or_scene *s, double *psi, double *grad) {
    if (!s->beta_air) {
        or_laplacian(s, s->beta, psi, grad);
        return;
    }
    const long nvox = nvox_of(s);
    double *a = (double *)malloc(sizeof(double) * nvox);
    for (long k = 0; k < nvox; ++k) a[k] = s->beta[k] - s->beta_air[k];
    or_laplacian(s, a, psi, grad);
    free(a);
}

/* ----------------------------------------------------------------------------------------- */
/* loss (Eq. Cost, one channel) and surrogate gradient with j fixed (Eq. Jaco1-DivTc)        */

enum { COND_NONE = 0, COND_INV_COUNT = 1, COND_COUNT = 2 };

static double residual(const or_scene *s, const double *img, const double *meas, const uint8_t *mask, double *rr) {
    long np = total_pixels(s);
    double E = 0.0;
    for (long p = 0; p < np; ++p) {
        double m = (mask && !mask[p]) ? 0.0 : 1.0;
        double r = m * (img[p] - meas[p]);
        E += r * r;
        rr[p] = 2.0 * r;   /* dE/di_c(p) */
    }
    return E;
}

/* beta is s->beta. L_ref, beta_ref define j = L_ref / beta_ref (0 where beta_ref = 0).
 * Outputs: img [sum W*H], grad [nvox], *loss. */
void or_surrogate_grad(const or_scene *s, const double *L_ref, const double *beta_ref, const double *meas,
                       const uint8_t *mask, int conditioning, double eta, double *img, double *grad, double *loss) {
    const long nvox = nvox_of(s), nL = (long)s->n_cams * nvox, np = total_pixels(s);
    double *j = (double *)malloc(sizeof(double) * nL);
    double *L = (double *)malloc(sizeof(double) * nL);
    double *T = (double *)malloc(sizeof(double) * nL);
    double *b = (double *)malloc(sizeof(double) * nL);
    double *sv = (double *)malloc(sizeof(double) * nL);
    double *gT = (double *)malloc(sizeof(double) * nL);
    double *Q = (double *)malloc(sizeof(double) * nL);
    double *rr = (double *)malloc(sizeof(double) * np);
    for (long i = 0; i < nL; ++i) {
        long k = i % nvox;
        j[i] = beta_ref[k] > 0 ? L_ref[i] / beta_ref[k] : 0.0;   /* Eq. Jc */
        L[i] = j[i] * s->beta[k];
    }
    or_transmittance(s, NULL, T);
    or_images(s, L, T, img);
    double E = residual(s, img, meas, mask, rr);
    or_backproject(s, rr, b);
    for (long i = 0; i < nL; ++i) sv[i] = L[i] * T[i] * b[i];
    or_los_adjoint(s, sv, gT);
    if (conditioning != COND_NONE) or_ray_counts(s, Q);
    for (long k = 0; k < nvox; ++k) {
        double g = 0.0;
        for (int c = 0; c < s->n_cams; ++c) {
            long i = (long)c * nvox + k;
            double q = 1.0;
            if (conditioning == COND_INV_COUNT) q = 1.0 / (Q[i] > 1.0 ? Q[i] : 1.0);
            else if (conditioning == COND_COUNT) q = Q[i];
            /* Q_c [ D{j} D{T} b  -  W^T (L T b) ]  (Eq. Jaco1, Eq. TcofJaco1, Eq. DivTc) */
            g += q * (j[i] * T[i] * b[i] - gT[i]);
        }
        grad[k] = g;
    }
    if (eta != 0.0) {
        double psi;
        double *gr = (double *)malloc(sizeof(double) * nvox);
        laplacian_of_aerosol(s, &psi, gr);
        E += eta * psi;
        for (long k = 0; k < nvox; ++k) grad[k] += eta * gr[k];
        free(gr);
    }
    *loss = E;
    free(j); free(L); free(T); free(b); free(sv); free(gT); free(Q); free(rr);
}

/* ----------------------------------------------------------------------------------------- */
/* full gradient: dE/dbeta = sum_c [ (dL_c/dbeta)^T a_c - W_c^T (L_c T_c b_c) ],            */
/* a_c = T_c b_c. dE[L]/dbeta by the score of the free-flight density: for every flight j   */
/* that ends in a collision, S_j = sum_{s>=j} w_s multiplies                                */
/*   -(length of flight j inside voxel m)  +  [m == k_j] / beta(k_j).                        */

/* Score part of the full gradient (Sec. 5 extended: the score of the free-flight density of
 * Eq. beer-lambert / Eq. MCextinct): every photon is replayed with its Philox key and records its
 * voxel segments and events; w_s is the event's contribution to <dE/di, i> through the
 * estimator (adj: voxel estimator, a_c(k) = T_c(k) b_c(k); cres: classic estimator, dE/di of
 * the pixel each camera sees the event in, plus the shadow-ray terms into the same sums);
 * S_j = sum_{s >= j} w_s; each flight j scatters -S_j * length into the voxels it crosses and
 * S_j / beta at its collision voxel. Adds into gout [nvox]. */
static void replay_score(const or_scene *s, const or_params *P, int nthreads, const double *adj, const double *cres,
                         const uint8_t *skip, double *gout) {
    const long nvox = nvox_of(s);
    int nt = nthreads_of(nthreads);
    double *accG = (double *)calloc((size_t)nt * nvox, sizeof(double));
    const long n = (long)P->n_photons;
#pragma omp parallel num_threads(nt)
    {
        int tid = 0;
#ifdef _OPENMP
        tid = omp_get_thread_num();
#endif
        double st_dummy[ST_N];
        double *g = accG + (size_t)tid * nvox;
        path_rec rec;
        memset(&rec, 0, sizeof(rec));
        tctx c;
        tctx_init(&c, s, P);
        c.stats = st_dummy;
        c.adj = adj;
        c.cres = cres;
        c.gsh = g;
        c.rec = &rec;
        double *S = NULL;
        long capS = 0;
#pragma omp for schedule(static, 4096)
        for (long i = 0; i < n; ++i) {
            if (skip && skip[i]) continue;
            rec.n_seg = 0;
            rec.n_ev = 0;
            trace_photon(&c, P->photon_offset + (uint64_t)i);
            if (rec.n_ev == 0) continue;
            if (rec.n_ev + 1 > capS) {
                capS = 2 * (rec.n_ev + 1);
                S = (double *)realloc(S, capS * sizeof(double));
            }
            /* suffix sums S_j, j = 1..n_ev */
            S[rec.n_ev] = 0.0;
            for (long e = rec.n_ev - 1; e >= 0; --e) S[e] = S[e + 1] + rec.ev_w[e];
            for (long q = 0; q < rec.n_seg; ++q) {
                int f = rec.flight_of_seg[q];          /* flight f ends at event f (if any) */
                if (f > rec.n_ev) continue;            /* final escaping flight: S = 0 */
                g[rec.seg_k[q]] -= S[f - 1] * rec.seg_len[q];
            }
            for (long e = 0; e < rec.n_ev; ++e) {
                /* collision density of the event's particle: beta_aerosol(k) for an aerosol
                 * event (score 1 / beta_aerosol), beta_air(k) for an air event (no beta_aerosol
                 * dependence) */
                long k = rec.ev_k[e];
                if (rec.ev_air[e]) continue;
                g[k] += S[e] / (s->beta[k] - (s->beta_air ? s->beta_air[k] : 0.0));
            }
        }
        free(S);
        free(rec.seg_k); free(rec.seg_len); free(rec.flight_of_seg); free(rec.ev_k); free(rec.ev_w);
        free(rec.ev_air);
    }
    for (long k = 0; k < nvox; ++k)
        for (int t = 0; t < nt; ++t) gout[k] += accG[(size_t)t * nvox + k];
    free(accG);
}

void or_full_grad(const or_scene *s, const or_params *P, const double *meas, const uint8_t *mask, double eta,
                  int nthreads, double *img, double *grad, double *loss, double *L_out, double *stats,
                  const uint8_t *skip) {
    const long nvox = nvox_of(s), nL = (long)s->n_cams * nvox, np = total_pixels(s);
    double *L = L_out ? L_out : (double *)malloc(sizeof(double) * nL);
    double *T = (double *)malloc(sizeof(double) * nL);
    double *b = (double *)malloc(sizeof(double) * nL);
    double *sv = (double *)malloc(sizeof(double) * nL);
    double *gT = (double *)malloc(sizeof(double) * nL);
    double *rr = (double *)malloc(sizeof(double) * np);
    double st_local[ST_N];
    const int prev_threads = threads_begin(nthreads);
    or_render(s, P, L, NULL, stats ? stats : st_local, NULL, skip, nthreads, NULL);
    or_transmittance(s, NULL, T);
    or_images(s, L, T, img);
    double E = residual(s, img, meas, mask, rr);
    or_backproject(s, rr, b);
    for (long i = 0; i < nL; ++i) sv[i] = L[i] * T[i] * b[i];
    or_los_adjoint(s, sv, gT);
    double *adj = (double *)malloc(sizeof(double) * nL);
    for (long i = 0; i < nL; ++i) adj[i] = T[i] * b[i];
    for (long k = 0; k < nvox; ++k) {
        double g = 0.0;
        for (int c = 0; c < s->n_cams; ++c) g -= gT[(long)c * nvox + k];
        grad[k] = g;
    }
    replay_score(s, P, nthreads, adj, NULL, skip, grad);
    if (eta != 0.0) {
        double psi;
        double *gr = (double *)malloc(sizeof(double) * nvox);
        laplacian_of_aerosol(s, &psi, gr);
        E += eta * psi;
        for (long k = 0; k < nvox; ++k) grad[k] += eta * gr[k];
        free(gr);
    }
    *loss = E;
    threads_end(prev_threads);
    free(adj);
    if (!L_out) free(L);
    free(T); free(b); free(sv); free(gT); free(rr);
}

/* Full gradient of the loss of the classic local estimate (Eq. fle): images by the forward
 * classic estimator, r = dE/di, then the score replay with w_s = sum_c r(p_c(s)) f_c(s), where
 * f_c(s) = albedo I_s P exp(-tau(X_s -> X_c)) / (|X_c - X_s|^2 Omega_p) is the event's
 * contribution to pixel p_c(s), plus each contribution's own dependence on beta through its
 * shadow ray, -r f * (length of the shadow ray in voxel m). */
void or_full_grad_classic(const or_scene *s, const or_params *P, const double *meas, const uint8_t *mask,
                          double eta, int nthreads, double *img, double *grad, double *loss, double *stats,
                          const uint8_t *skip) {
    const long nvox = nvox_of(s), np = total_pixels(s);
    double *rr = (double *)malloc(sizeof(double) * np);
    double st_local[ST_N];
    for (long p = 0; p < np; ++p) img[p] = 0.0;
    or_render(s, P, NULL, img, stats ? stats : st_local, NULL, skip, nthreads, NULL);
    double E = residual(s, img, meas, mask, rr);
    for (long k = 0; k < nvox; ++k) grad[k] = 0.0;
    replay_score(s, P, nthreads, NULL, rr, skip, grad);
    if (eta != 0.0) {
        double psi;
        double *gr = (double *)malloc(sizeof(double) * nvox);
        laplacian_of_aerosol(s, &psi, gr);
        E += eta * psi;
        for (long k = 0; k < nvox; ++k) grad[k] += eta * gr[k];
        free(gr);
    }
    *loss = E;
    free(rr);
}

/* ----------------------------------------------------------------------------------------- */
/* backward MC with the sun local estimate (Eq. ble), one pixel: checks Helmholtz            */
/* reciprocity against the forward estimates and is the reference of the GPU BMC. The pixel  */
/* is sampled uniformly on the image plane and weighted by cos^3 * A_pix / Omega_p, so the   */
/* mean is the pixel's solid-angle average radiance. A point is sunlit only if its sun-ward  */
/* ray leaves through the top face, matching top-face illumination in the forward model.     */
/* Sample q of global pixel p draws Philox counters (q, event, 1 + p): every pixel has its   */
/* own stream (the forward transport uses stream word 0).                                    */

void or_bmc_pixel(const or_scene *s, const or_params *P, int c, int i, int j, uint64_t n, double *mean, double *var) {
    double sun[3] = {-sin(P->sun_zenith) * cos(P->sun_azimuth), -sin(P->sun_zenith) * sin(P->sun_azimuth),
                     -cos(P->sun_zenith)};
    double to_sun[3] = {-sun[0], -sun[1], -sun[2]};
    double tx, ty;
    cam_tan(s, c, &tx, &ty);
    const int W = s->cam_w[c], H = s->cam_h[c];
    double x1 = (2.0 * i / W - 1.0) * tx, x2 = (2.0 * (i + 1) / W - 1.0) * tx;
    double y1 = (2.0 * j / H - 1.0) * ty, y2 = (2.0 * (j + 1) / H - 1.0) * ty;
    double omega = rect_solid_angle(x1, x2, y1, y2);
    double apix = (x2 - x1) * (y2 - y1);
    const double *Pc = s->cam_pos + 3 * c;
    const uint32_t stream = (uint32_t)(1 + pix_offset(s, c) + (long)j * W + i);
    double sum = 0.0, sum2 = 0.0;
    double st[ST_N];
    tctx cx;
    tctx_init(&cx, s, P);
    cx.stats = st;
    for (uint64_t q = 0; q < n; ++q) {
        double u[4];
        draws4(P->seed, q, 0, stream, u);
        double px = i + u[0], py = j + u[1];
        double xx = (2.0 * px / W - 1.0) * tx, yy = (2.0 * py / H - 1.0) * ty;
        double cosv = 1.0 / sqrt(1.0 + xx * xx + yy * yy);
        double wpix = cosv * cosv * cosv * apix / omega;
        double d[3], t0;
        int v[3];
        pixel_dir(s, c, px, py, d);
        double contrib = 0.0;
        if (ray_enter(s, Pc, d, v, &t0)) {
            double X[3] = {Pc[0] + t0 * d[0], Pc[1] + t0 * d[1], Pc[2] + t0 * d[2]};
            double I = 1.0, tau = -log(1.0 - u[2]);
            for (uint32_t ev = 1;; ++ev) {
                double Xn[3];
                int vn[3], face;
                if (!flight(&cx, X, d, v, tau, Xn, vn, &face, 0)) break;
                /* local estimate toward the sun */
                tau_ctx tc = {s->beta, 0.0};
                int exitf = walk(s, Xn, to_sun, vn, 0.0, INFINITY, tau_visit, &tc);
                double mu = d[0] * to_sun[0] + d[1] * to_sun[1] + d[2] * to_sun[2];
                if (exitf == 5) contrib += P->albedo * I * or_hg_phase(P->g, mu) * exp(-tc.tau) * P->sun_irradiance;
                I *= P->albedo;
                if (I == 0.0) break;
                if (P->max_order > 0 && (int)ev >= P->max_order) break;
                if ((int)ev >= P->max_events) break;
                draws4(P->seed, q, ev, stream, u);
                if (I < P->rr_threshold) {
                    if (u[2] < P->rr_survival) I /= P->rr_survival;
                    else break;
                }
                double ct = or_hg_sample(P->g, u[0]), nd[3];
                or_rotate(d, ct, 2.0 * OR_PI * u[1], nd);
                for (int a = 0; a < 3; ++a) { X[a] = Xn[a]; d[a] = nd[a]; v[a] = vn[a]; }
                tau = -log(1.0 - u[3]);
            }
        }
        double val = contrib * wpix;
        sum += val;
        sum2 += val * val;
    }
    *mean = sum / n;
    *var = (sum2 / n - (*mean) * (*mean)) / (n > 1 ? (n - 1) : 1);   /* variance of the mean */
}

int or_version(void) { return 1; }
