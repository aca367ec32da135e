/*
 * gs_oracle.c -- plain FP64 CPU oracle for stochastic ray tracing of
 * transparent 3D Gaussians (arXiv 2504.06598).
 *
 * TEST INFRASTRUCTURE ONLY. Only the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load this library. The CUDA path
 * never calls it and shares no code, header or constant table with it.
 *
 * Everything here is a direct, slow restatement of the paper's definitions:
 * every ray is tested against every Gaussian (no acceleration structure),
 * all per-candidate arithmetic is double precision, and the exact sorted
 * blend is computed by collecting and sorting all valid intersections.
 *
 *   Eq. 1   Gaussian G(x) = exp(-1/2 (x-mu)^T Sigma^-1 (x-mu)),
 *           Sigma = R^T S^2 R  (R maps world to local).
 *   Eq. 2   bounding ellipsoid ||S^-1 R (x-mu)|| <= s, s = 2 sqrt(2).
 *   Sec. 3.1  the ray/Gaussian intersection is a 1D Gaussian along the ray;
 *           its mean is the shading depth; culled behind the origin or
 *           outside the bounding ellipsoid.
 *   Eq. 3   L = sum_i T_i alpha_i c_i, T_i = prod_{j<i} (1 - alpha_j).
 *   Eq. 4-6 binary opacities; the estimate is the colour of the closest
 *           accepted intersection.
 *   Eq. 7   mean of N estimates.
 *   Alg. 1  range test, negligibility test, random acceptance, clip.
 *
 * Readings of points the paper leaves open (listed in the design notes):
 *   - acceptance is xi < alpha (Fig. 2 and Eq. 4; Alg. 1 prints the test
 *     inverted);
 *   - alpha is the opacity times the peak of the 1D Gaussian along the ray,
 *     alpha = o * exp(-q/2) with q the minimum of the quadratic form on the
 *     ray (Fig. 2 caption: opacity at the mean of a 1D Gaussian);
 *   - the random draw is Philox-4x32-10 (Salmon et al., SC'11) keyed by
 *     seed, with counter (ray_id, gid, sample >> 2, stream_tag) and lane
 *     sample & 3, xi = (u >> 8) * 2^-24;
 *   - the quaternion (w,x,y,z) is normalised and gives R_q (local to world),
 *     the paper's R is R_q^T, so Sigma = R_q S^2 R_q^T;
 *   - candidates are ordered by (t, gid) lexicographically, so equal depths
 *     resolve to the smaller Gaussian id, in the estimator and the blend;
 *   - the colour is c = max(0, k_0 + sum_{l>=1,m} Y_lm(d) k_lm) with the DC
 *     coefficient stored pre-multiplied, real spherical harmonics with the
 *     Condon-Shortley phase, d the unit ray direction;
 *   - camera rays are defined as float32 values computed by a fixed sequence
 *     of correctly rounded float operations (see orc_camera_ray); every
 *     later step promotes them to double.
 *
 * Pins: every function is checked by the -m "not gpu" tests against values
 * the paper prints, closed forms, invariants, brute force or library
 * routines.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_S2 8.0 /* s^2 with s = 2*sqrt(2) (Eq. 2) */

typedef struct {
    int64_t M;
    const float *means;          /* [M][3] */
    const float *log_scales;     /* [M][3] */
    const float *quats;          /* [M][4] w,x,y,z */
    const float *opacity_logits; /* [M] */
    const float *sh;             /* [M][K][3] */
    int32_t sh_degree;
    int32_t pad;
} orc_scene;

typedef struct {
    float eye[3];
    float look_at[3];
    float up[3];
    float fov_y_deg;
    int32_t width;
    int32_t height;
    uint32_t ray_id_offset;
    int32_t pad;
} orc_pinhole;

typedef struct {
    uint64_t seed;
    int32_t spp;
    int32_t n_hits;
    double t_min;
    double t_max;
    double bg[3];
    uint32_t stream_tag;
    int32_t depth_mode; /* 0: mean of the 1D Gaussian; 1: projected centre */
    int32_t rng_mode;   /* 0: Philox; 1: trigonometric hash of the hit point */
    int32_t pad;
} orc_params;

/* ------------------------------------------------------------------ */
/* Philox-4x32-10, from Salmon, Moraes, Dror and Shaw, "Parallel random  */
/* numbers: as easy as 1, 2, 3" (SC'11): ten rounds of the Philox S-box  */
/* with multipliers 0xD2511F53 / 0xCD9E8D57 and Weyl key increments      */
/* 0x9E3779B9 / 0xBB67AE85 applied between rounds.                       */
/* ------------------------------------------------------------------ */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)x0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)x2;
        uint32_t y0 = (uint32_t)(p1 >> 32) ^ x1 ^ k0;
        uint32_t y1 = (uint32_t)p1;
        uint32_t y2 = (uint32_t)(p0 >> 32) ^ x3 ^ k1;
        uint32_t y3 = (uint32_t)p0;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* The uniform draw xi in [0,1) for (ray, Gaussian, sample). */
double orc_xi(uint64_t seed, uint32_t ray_id, uint32_t gid, uint32_t sample, uint32_t stream_tag)
{
    uint32_t ctr[4] = {ray_id, gid, sample >> 2, stream_tag};
    uint32_t key[2] = {(uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32)};
    uint32_t u[4];
    orc_philox4x32_10(ctr, key, u);
    return (double)(u[sample & 3u] >> 8) * (1.0 / 16777216.0);
}

/* Trigonometric hash of a hit position (Sec. 4.2, Eq. 8-9):
 *   r1(q) = fract(b1 sin(a1 q)), r2(q) = fract(b2 sin(a2^T q)),
 *   xi(p) = r2(p_xy + r1(p_z)),
 * with the coefficients the paper states after Eq. 9 (below). Both entries
 * of b2 are equal, so both components of r2 are equal; the first is used.
 * The paper makes the draws change between frames by jittering the camera
 * rays; here the rays are fixed, so sample s hashes p + delta_s, with
 * delta_s = 1e-3 * (frac(s c1), frac(s c2), frac(s c3)) - 5e-4 from the
 * additive recurrence with c = (0.8191725134, 0.6710436067, 0.5497004779).
 * The coefficients are pinned to the paper's printed values; the paper
 * prints no hash values, so the composition is pinned through points where
 * every sine is 0 or 1 (the draw is then a known fraction) and through the
 * invariances the composition implies. */
static const double kHashA1 = 91.3458;
static const double kHashB1 = 47453.5453;
static const double kHashA2[2] = {12.9898, 78.233};
static const double kHashB2[2] = {43758.5453, 43758.5453};

/* The coefficients orc_hash_xi uses: a1, b1, a2[0], a2[1], b2[0], b2[1]. */
void orc_hash_constants(double out[6])
{
    out[0] = kHashA1;
    out[1] = kHashB1;
    out[2] = kHashA2[0];
    out[3] = kHashA2[1];
    out[4] = kHashB2[0];
    out[5] = kHashB2[1];
}

static double fract_d(double x) { return x - floor(x); }

double orc_hash_xi(const double p[3], uint32_t sample)
{
    const double c[3] = {0.8191725134, 0.6710436067, 0.5497004779};
    double q[3];
    for (int i = 0; i < 3; ++i) q[i] = p[i] + 1e-3 * fract_d((double)sample * c[i]) - 5e-4;
    double r1 = fract_d(kHashB1 * sin(kHashA1 * q[2]));
    double x = q[0] + r1, y = q[1] + r1;
    return fract_d(kHashB2[0] * sin(kHashA2[0] * x + kHashA2[1] * y));
}

/* Camera forward axis of a pinhole, float32 as in orc_camera_ray. */
static void cam_forward(const float eye[3], const float at[3], double f[3]);

/* ------------------------------------------------------------------ */
/* Parameter activation (Eq. 1)                                          */
/* ------------------------------------------------------------------ */

/* Rotation matrix (row-major, local to world) of the normalised
 * quaternion (w,x,y,z). */
static void quat_to_rot(const float *qf, double R[9])
{
    double w = qf[0], x = qf[1], y = qf[2], z = qf[3];
    double n = sqrt(w * w + x * x + y * y + z * z);
    w /= n; x /= n; y /= n; z /= n;
    R[0] = 1.0 - 2.0 * (y * y + z * z);
    R[1] = 2.0 * (x * y - w * z);
    R[2] = 2.0 * (x * z + w * y);
    R[3] = 2.0 * (x * y + w * z);
    R[4] = 1.0 - 2.0 * (x * x + z * z);
    R[5] = 2.0 * (y * z - w * x);
    R[6] = 2.0 * (x * z - w * y);
    R[7] = 2.0 * (y * z + w * x);
    R[8] = 1.0 - 2.0 * (x * x + y * y);
}

typedef struct {
    double mu[3];
    double Sinv[9]; /* Sigma^-1, row-major, symmetric */
    double opacity;
} orc_gauss;

static void activate_one(const orc_scene *sc, int64_t g, orc_gauss *out)
{
    double R[9];
    quat_to_rot(sc->quats + 4 * g, R);
    double inv_s2[3];
    for (int k = 0; k < 3; ++k) {
        double s = exp((double)sc->log_scales[3 * g + k]);
        inv_s2[k] = 1.0 / (s * s);
    }
    /* Sigma^-1 = R_q S^-2 R_q^T */
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double acc = 0.0;
            for (int k = 0; k < 3; ++k)
                acc += R[3 * i + k] * inv_s2[k] * R[3 * j + k];
            out->Sinv[3 * i + j] = acc;
        }
    for (int k = 0; k < 3; ++k)
        out->mu[k] = (double)sc->means[3 * g + k];
    out->opacity = 1.0 / (1.0 + exp(-(double)sc->opacity_logits[g]));
}

/* Exported for tests: opacity [M], R_q [M][9], Sigma^-1 [M][9]. */
void orc_activate(const orc_scene *sc, double *opacity, double *rot, double *sigma_inv)
{
    for (int64_t g = 0; g < sc->M; ++g) {
        orc_gauss a;
        activate_one(sc, g, &a);
        if (opacity) opacity[g] = a.opacity;
        if (rot) quat_to_rot(sc->quats + 4 * g, rot + 9 * g);
        if (sigma_inv) memcpy(sigma_inv + 9 * g, a.Sinv, sizeof a.Sinv);
    }
}

/* ------------------------------------------------------------------ */
/* 1D Gaussian along the ray (Sec. 3.1, Alg. 1 GetGauss1D)               */
/* Along x(t) = o + t d the exponent is (a t^2 + 2 b t + c) / 2 with     */
/* a = d^T Sinv d, b = d^T Sinv (o-mu), c = (o-mu)^T Sinv (o-mu).       */
/* Its mean is t* = -b/a and the minimum of the quadratic form is        */
/* q = c - b^2/a, so the peak of the 1D Gaussian is exp(-q/2).           */
/* ------------------------------------------------------------------ */
static void gauss1d(const orc_gauss *G, const double o[3], const double d[3], double *t, double *q)
{
    double op[3] = {o[0] - G->mu[0], o[1] - G->mu[1], o[2] - G->mu[2]};
    double Sd[3], So[3];
    for (int i = 0; i < 3; ++i) {
        Sd[i] = G->Sinv[3 * i + 0] * d[0] + G->Sinv[3 * i + 1] * d[1] + G->Sinv[3 * i + 2] * d[2];
        So[i] = G->Sinv[3 * i + 0] * op[0] + G->Sinv[3 * i + 1] * op[1] + G->Sinv[3 * i + 2] * op[2];
    }
    double a = d[0] * Sd[0] + d[1] * Sd[1] + d[2] * Sd[2];
    double b = d[0] * So[0] + d[1] * So[1] + d[2] * So[2];
    double c = op[0] * So[0] + op[1] * So[1] + op[2] * So[2];
    *t = -b / a;
    double qq = c - b * b / a;
    *q = qq > 0.0 ? qq : 0.0;
}

/* Exported for tests: evaluate Gaussian g against one ray.
 * out = {t*, q, alpha, valid}. */
void orc_eval_pair(const orc_scene *sc, int64_t g, const double o[3], const double d[3],
                   double t_min, double t_max, double out[4])
{
    orc_gauss G;
    activate_one(sc, g, &G);
    double t, q;
    gauss1d(&G, o, d, &t, &q);
    out[0] = t;
    out[1] = q;
    out[2] = G.opacity * exp(-0.5 * q);
    out[3] = (t > t_min && t < t_max && q <= ORC_S2) ? 1.0 : 0.0;
}

/* ------------------------------------------------------------------ */
/* Real spherical harmonics (Condon-Shortley phase), built from the      */
/* associated Legendre functions by the standard three-term recursion.   */
/* Index K = l*l + l + m, m = -l..l.                                     */
/* ------------------------------------------------------------------ */
static double factorial(int n)
{
    double f = 1.0;
    for (int i = 2; i <= n; ++i) f *= i;
    return f;
}

/* Associated Legendre P_l^m(z), m >= 0, including the (-1)^m phase. */
static double assoc_legendre(int l, int m, double z)
{
    double somx2 = sqrt((1.0 - z) * (1.0 + z));
    double pmm = 1.0; /* P_m^m = (-1)^m (2m-1)!! (1-z^2)^{m/2} */
    double fact = 1.0;
    for (int i = 1; i <= m; ++i) {
        pmm *= -fact * somx2;
        fact += 2.0;
    }
    if (l == m) return pmm;
    double pmmp1 = z * (2.0 * m + 1.0) * pmm; /* P_{m+1}^m */
    if (l == m + 1) return pmmp1;
    double pll = 0.0;
    for (int ll = m + 2; ll <= l; ++ll) {
        pll = ((2.0 * ll - 1.0) * z * pmmp1 - (ll + m - 1.0) * pmm) / (ll - m);
        pmm = pmmp1;
        pmmp1 = pll;
    }
    return pll;
}

/* Exported: Y[K] for K = 0..(deg+1)^2-1 at unit direction d. */
void orc_sh_basis(int deg, const double d[3], double *Y)
{
    double z = d[2];
    if (z > 1.0) z = 1.0;
    if (z < -1.0) z = -1.0;
    double phi = atan2(d[1], d[0]);
    for (int l = 0; l <= deg; ++l) {
        for (int m = -l; m <= l; ++m) {
            int am = m < 0 ? -m : m;
            double K = sqrt((2.0 * l + 1.0) / (4.0 * M_PI) * factorial(l - am) / factorial(l + am));
            double P = assoc_legendre(l, am, z);
            double v;
            if (m == 0)
                v = K * P;
            else if (m > 0)
                v = sqrt(2.0) * K * P * cos(am * phi);
            else
                v = sqrt(2.0) * K * P * sin(am * phi);
            Y[l * l + l + m] = v;
        }
    }
}

/* Colour of Gaussian g seen along unit direction d (DC pre-multiplied). */
static void sh_colour(const orc_scene *sc, int64_t g, const double *Y, double rgb[3])
{
    int K = (sc->sh_degree + 1) * (sc->sh_degree + 1);
    const float *k = sc->sh + (size_t)g * K * 3;
    for (int ch = 0; ch < 3; ++ch) {
        double acc = (double)k[ch];
        for (int i = 1; i < K; ++i) acc += Y[i] * (double)k[3 * i + ch];
        rgb[ch] = acc > 0.0 ? acc : 0.0;
    }
}

/* ------------------------------------------------------------------ */
/* Camera rays, defined in float32. With fov in degrees:                 */
/*   th = (float) tan(fov * pi / 360)               (double, then float) */
/*   f  = normalise(look_at - eye), r = normalise(f x up), u = r x f     */
/*   s  = th / H                                                         */
/*   ux = (2x + 1 - W) * s,  uy = (H - 1 - 2y) * s                       */
/*   d  = normalise((f + ux r) + uy u),  o = eye                         */
/* with normalise(v) = v / sqrt((vx*vx + vy*vy) + vz*vz), every product, */
/* sum, quotient and square root rounded once to float.                  */
/* ------------------------------------------------------------------ */
static void normalise_f(float v[3])
{
    float n2 = v[0] * v[0];
    n2 = n2 + v[1] * v[1];
    n2 = n2 + v[2] * v[2];
    float n = sqrtf(n2);
    v[0] = v[0] / n;
    v[1] = v[1] / n;
    v[2] = v[2] / n;
}

static void cross_f(const float a[3], const float b[3], float c[3])
{
    float p, m;
    p = a[1] * b[2]; m = a[2] * b[1]; c[0] = p - m;
    p = a[2] * b[0]; m = a[0] * b[2]; c[1] = p - m;
    p = a[0] * b[1]; m = a[1] * b[0]; c[2] = p - m;
}

static void cam_forward(const float eye[3], const float at[3], double f[3])
{
    float ff[3];
    for (int i = 0; i < 3; ++i) ff[i] = at[i] - eye[i];
    normalise_f(ff);
    for (int i = 0; i < 3; ++i) f[i] = (double)ff[i];
}

void orc_camera_ray(const orc_pinhole *cam, int32_t x, int32_t y, double o[3], double d[3],
                    uint32_t *ray_id)
{
    float f[3], r[3], u[3], dr[3];
    for (int i = 0; i < 3; ++i) f[i] = cam->look_at[i] - cam->eye[i];
    normalise_f(f);
    cross_f(f, cam->up, r);
    normalise_f(r);
    cross_f(r, f, u);
    float th = (float)tan((double)cam->fov_y_deg * 3.14159265358979323846 / 360.0);
    float s = th / (float)cam->height;
    float ux = (float)(2 * x + 1 - cam->width) * s;
    float uy = (float)(cam->height - 1 - 2 * y) * s;
    for (int i = 0; i < 3; ++i) {
        float a = ux * r[i];
        float b = uy * u[i];
        float c = f[i] + a;
        dr[i] = c + b;
    }
    normalise_f(dr);
    for (int i = 0; i < 3; ++i) {
        o[i] = (double)cam->eye[i];
        d[i] = (double)dr[i];
    }
    if (ray_id) *ray_id = cam->ray_id_offset + (uint32_t)y * (uint32_t)cam->width + (uint32_t)x;
}

/* ------------------------------------------------------------------ */
/* Candidates, payload update, blend, enumeration                        */
/* ------------------------------------------------------------------ */
typedef struct {
    double t, q, alpha;
    double rgb[3];
    int32_t gid;
} orc_cand;

static int lex_less(double ta, int32_t ga, double tb, int32_t gb)
{
    return ta < tb || (ta == tb && ga < gb);
}

static int cand_cmp(const void *pa, const void *pb)
{
    const orc_cand *a = (const orc_cand *)pa, *b = (const orc_cand *)pb;
    if (lex_less(a->t, a->gid, b->t, b->gid)) return -1;
    if (lex_less(b->t, b->gid, a->t, a->gid)) return 1;
    return 0;
}

/* Fig. 2 / Eq. 6: process candidates in the given order, replacing the
 * payload whenever an accepted candidate is closer than the stored one.
 * Returns the index of the winner, or -1. */
int64_t orc_closest_accepted(int64_t n, const double *t, const int32_t *gid,
                             const uint8_t *accepted, const int64_t *order)
{
    int64_t win = -1;
    for (int64_t k = 0; k < n; ++k) {
        int64_t i = order ? order[k] : k;
        if (!accepted[i]) continue;
        if (win < 0 || lex_less(t[i], gid[i], t[win], gid[win])) win = i;
    }
    return win;
}

/* Eq. 3 with background: candidates are sorted by (t, gid) first. The
 * optional second output is the same composite of squared colours, which is
 * E[L^2] of the single-sample estimate of Eq. 6: sample s returns c_i with
 * probability T_i alpha_i and bg with probability T_{M+1}. */
static void blend_sorted(int64_t n, const orc_cand *c, const double bg[3], double out[3],
                         double *out2)
{
    double T = 1.0;
    double L[3] = {0.0, 0.0, 0.0};
    double L2[3] = {0.0, 0.0, 0.0};
    for (int64_t i = 0; i < n; ++i) {
        for (int ch = 0; ch < 3; ++ch) {
            L[ch] += T * c[i].alpha * c[i].rgb[ch];
            L2[ch] += T * c[i].alpha * c[i].rgb[ch] * c[i].rgb[ch];
        }
        T *= (1.0 - c[i].alpha);
    }
    for (int ch = 0; ch < 3; ++ch) {
        out[ch] = L[ch] + T * bg[ch];
        if (out2) out2[ch] = L2[ch] + T * bg[ch] * bg[ch];
    }
}

/* Exported: Eq. 3 on arbitrary (unsorted) candidate arrays. */
void orc_blend(int64_t n, const double *t, const int32_t *gid, const double *alpha,
               const double *rgb, const double bg[3], double out[3], double *out2)
{
    orc_cand *c = (orc_cand *)malloc((size_t)(n > 0 ? n : 1) * sizeof(orc_cand));
    for (int64_t i = 0; i < n; ++i) {
        c[i].t = t[i];
        c[i].gid = gid[i];
        c[i].alpha = alpha[i];
        for (int ch = 0; ch < 3; ++ch) c[i].rgb[ch] = rgb[3 * i + ch];
    }
    qsort(c, (size_t)n, sizeof(orc_cand), cand_cmp);
    blend_sorted(n, c, bg, out, out2);
    free(c);
}

/* Exported: expectation of Eq. 6 by enumerating all 2^n acceptance
 * vectors of n <= 24 candidates given in depth order. */
int orc_enumerate_expectation(int n, const double *alpha, const double *rgb, const double bg[3],
                              double out[3])
{
    if (n < 0 || n > 24) return -1;
    out[0] = out[1] = out[2] = 0.0;
    uint32_t total = 1u << n;
    for (uint32_t mask = 0; mask < total; ++mask) {
        double p = 1.0;
        for (int i = 0; i < n; ++i) p *= (mask >> i & 1u) ? alpha[i] : (1.0 - alpha[i]);
        int first = -1;
        for (int i = 0; i < n; ++i)
            if (mask >> i & 1u) { first = i; break; }
        for (int ch = 0; ch < 3; ++ch) out[ch] += p * (first >= 0 ? rgb[3 * first + ch] : bg[ch]);
    }
    return 0;
}

/* ------------------------------------------------------------------ */
/* Brute force over every Gaussian for one ray                           */
/* ------------------------------------------------------------------ */
typedef struct {
    orc_cand *v;
    int64_t n, cap;
} cand_list;

static void cand_push(cand_list *L, const orc_cand *c)
{
    if (L->n == L->cap) {
        L->cap = L->cap ? 2 * L->cap : 256;
        L->v = (orc_cand *)realloc(L->v, (size_t)L->cap * sizeof(orc_cand));
    }
    L->v[L->n++] = *c;
}

/* fwd != NULL: depth is the Gaussian centre projected on the camera's
 * forward axis (Sec. 4.1); alpha stays the peak of the 1D Gaussian. */
static void collect_mode(const orc_scene *sc, const orc_gauss *act, const double o[3],
                         const double d[3], double t_min, double t_max, const double *fwd,
                         cand_list *L)
{
    double Y[16];
    orc_sh_basis(sc->sh_degree, d, Y);
    L->n = 0;
    for (int64_t g = 0; g < sc->M; ++g) {
        double t, q;
        gauss1d(&act[g], o, d, &t, &q);
        if (fwd)
            t = (act[g].mu[0] - o[0]) * fwd[0] + (act[g].mu[1] - o[1]) * fwd[1] +
                (act[g].mu[2] - o[2]) * fwd[2];
        if (!(t > t_min && t < t_max)) continue; /* Alg. 1 range test */
        if (!(q <= ORC_S2)) continue;            /* Eq. 2 negligibility */
        orc_cand c;
        c.t = t;
        c.q = q;
        c.alpha = act[g].opacity * exp(-0.5 * q);
        c.gid = (int32_t)g;
        sh_colour(sc, g, Y, c.rgb);
        cand_push(L, &c);
    }
}

static void collect(const orc_scene *sc, const orc_gauss *act, const double o[3], const double d[3],
                    double t_min, double t_max, cand_list *L)
{
    collect_mode(sc, act, o, d, t_min, t_max, NULL, L);
}

static orc_gauss *activate_all(const orc_scene *sc)
{
    orc_gauss *act = (orc_gauss *)malloc((size_t)(sc->M > 0 ? sc->M : 1) * sizeof(orc_gauss));
    for (int64_t g = 0; g < sc->M; ++g) activate_one(sc, g, &act[g]);
    return act;
}

/* Exported: every valid candidate of one ray, in Gaussian-id order.
 * Arrays have room for cap entries; returns the number of candidates
 * (which may exceed cap, in which case only cap are written). */
int64_t orc_ray_candidates(const orc_scene *sc, const double o[3], const double d[3], double t_min,
                           double t_max, int64_t cap, double *t, double *q, double *alpha,
                           int32_t *gid, double *rgb)
{
    orc_gauss *act = activate_all(sc);
    cand_list L = {0, 0, 0};
    collect(sc, act, o, d, t_min, t_max, &L);
    for (int64_t i = 0; i < L.n && i < cap; ++i) {
        if (t) t[i] = L.v[i].t;
        if (q) q[i] = L.v[i].q;
        if (alpha) alpha[i] = L.v[i].alpha;
        if (gid) gid[i] = L.v[i].gid;
        if (rgb) for (int ch = 0; ch < 3; ++ch) rgb[3 * i + ch] = L.v[i].rgb[ch];
    }
    int64_t n = L.n;
    free(L.v);
    free(act);
    return n;
}

/* One ray: exact blend (Eq. 3) and S = spp*N estimator samples (Eq. 6),
 * averaged (Eq. 7). Sample s uses draw xi(seed, ray_id, gid, s). */
static void trace_one(const orc_scene *sc, const orc_gauss *act, const orc_params *p,
                      const double o[3], const double d[3], uint32_t ray_id, const double *fwd,
                      cand_list *L, double blend[3], double *blend2, double est[3],
                      int32_t *hit_id, double *hit_t)
{
    collect_mode(sc, act, o, d, p->t_min, p->t_max, p->depth_mode == 1 ? fwd : NULL, L);
    int64_t S = (int64_t)p->spp * p->n_hits;
    double acc[3] = {0.0, 0.0, 0.0};
    for (int64_t s = 0; s < S; ++s) {
        int64_t win = -1;
        for (int64_t i = 0; i < L->n; ++i) {
            double xi;
            if (p->rng_mode == 1) {
                double ph[3];
                for (int k = 0; k < 3; ++k) ph[k] = o[k] + L->v[i].t * d[k];
                xi = orc_hash_xi(ph, (uint32_t)s);
            } else {
                xi = orc_xi(p->seed, ray_id, (uint32_t)L->v[i].gid, (uint32_t)s, p->stream_tag);
            }
            if (!(xi < L->v[i].alpha)) continue; /* Eq. 4: accepted with probability alpha */
            if (win < 0 || lex_less(L->v[i].t, L->v[i].gid, L->v[win].t, L->v[win].gid)) win = i;
        }
        for (int ch = 0; ch < 3; ++ch) acc[ch] += win >= 0 ? L->v[win].rgb[ch] : p->bg[ch];
        if (hit_id) hit_id[s] = win >= 0 ? L->v[win].gid : -1;
        if (hit_t) hit_t[s] = win >= 0 ? L->v[win].t : INFINITY;
    }
    if (est)
        for (int ch = 0; ch < 3; ++ch) est[ch] = S > 0 ? acc[ch] / (double)S : 0.0;
    if (blend) {
        qsort(L->v, (size_t)L->n, sizeof(orc_cand), cand_cmp);
        blend_sorted(L->n, L->v, p->bg, blend, blend2);
    }
}

int orc_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Exported: render the listed pixels of a pinhole camera.
 * pix[i] = y*W + x. Outputs (each nullable):
 *   blend [n][3], est [n][3], hit_id [n][S], hit_t [n][S], n_valid [n].
 * Returns the number of threads used. */
int orc_render_pinhole(const orc_scene *sc, const orc_pinhole *cam, const orc_params *p,
                       int64_t n_pix, const int64_t *pix, double *blend, double *blend2,
                       double *est, int32_t *hit_id, double *hit_t, int64_t *n_valid,
                       int n_threads)
{
    orc_gauss *act = activate_all(sc);
    int64_t S = (int64_t)p->spp * p->n_hits;
    int used = 1;
#ifdef _OPENMP
    if (n_threads <= 0) n_threads = omp_get_max_threads();
#pragma omp parallel num_threads(n_threads)
#endif
    {
#ifdef _OPENMP
#pragma omp single
        used = omp_get_num_threads();
#endif
        cand_list L = {0, 0, 0};
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 4)
#endif
        for (int64_t i = 0; i < n_pix; ++i) {
            int32_t x = (int32_t)(pix[i] % cam->width), y = (int32_t)(pix[i] / cam->width);
            double o[3], d[3];
            uint32_t rid;
            orc_camera_ray(cam, x, y, o, d, &rid);
            double fwd[3];
            cam_forward(cam->eye, cam->look_at, fwd);
            trace_one(sc, act, p, o, d, rid, fwd, &L, blend ? blend + 3 * i : 0,
                      blend2 ? blend2 + 3 * i : 0, est ? est + 3 * i : 0,
                      hit_id ? hit_id + S * i : 0, hit_t ? hit_t + S * i : 0);
            if (n_valid) n_valid[i] = L.n;
        }
        free(L.v);
    }
    free(act);
    return used;
}

/* Exported: same for explicit rays (origins/dirs given as float32 values,
 * dirs of unit length), ray_ids[i] keys the draws of ray i. */
int orc_render_rays(const orc_scene *sc, const orc_params *p, int64_t n_rays, const float *origins,
                    const float *dirs, const uint32_t *ray_ids, double *blend, double *blend2,
                    double *est, int32_t *hit_id, double *hit_t, int64_t *n_valid,
                    int n_threads)
{
    orc_gauss *act = activate_all(sc);
    int64_t S = (int64_t)p->spp * p->n_hits;
    int used = 1;
#ifdef _OPENMP
    if (n_threads <= 0) n_threads = omp_get_max_threads();
#pragma omp parallel num_threads(n_threads)
#endif
    {
#ifdef _OPENMP
#pragma omp single
        used = omp_get_num_threads();
#endif
        cand_list L = {0, 0, 0};
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 4)
#endif
        for (int64_t i = 0; i < n_rays; ++i) {
            double o[3], d[3];
            for (int k = 0; k < 3; ++k) {
                o[k] = (double)origins[3 * i + k];
                d[k] = (double)dirs[3 * i + k];
            }
            trace_one(sc, act, p, o, d, ray_ids[i], NULL, &L, blend ? blend + 3 * i : 0,
                      blend2 ? blend2 + 3 * i : 0, est ? est + 3 * i : 0,
                      hit_id ? hit_id + S * i : 0, hit_t ? hit_t + S * i : 0);
            if (n_valid) n_valid[i] = L.n;
        }
        free(L.v);
    }
    free(act);
    return used;
}

/* ------------------------------------------------------------------ */
/* Gradients (the paper's closing remark on differentiable rendering,  */
/* Sec. 6). For a scalar G = sum_rays g . L with g the given per-ray     */
/* weight (dLoss/dL), parameters theta_i = (mu[3], log_s[3], quat[4],    */
/* logit) and SH coefficients k_i of every Gaussian.                     */
/*                                                                       */
/* alpha = o exp(-q/2), o = sigmoid(logit), q = v^T Sigma^-1 v with      */
/* v = o_ray + t* d - mu at the 1D mean t* (dq/dt = 0 there, so t* is    */
/* held fixed when differentiating q). Sigma^-1 = R S^-2 R^T with R the   */
/* rotation of the normalised quaternion.                                */
/*                                                                       */
/* Exact blend (Eq. 3): dL/dalpha_i = T_i (c_i - B_i), B_i the blend of   */
/* everything behind i including the background; dL/dc_i = T_i alpha_i.  */
/* Stochastic estimate (one sample with closest accepted hit k, colour   */
/* c_k or bg): dL/dc_k = 1, and for every valid i in front of k          */
/* dL/dalpha_i = (c_i - c_k) / (1 - alpha_i). Both are unbiased for the  */
/* blend gradient: i in front of k means i and its prefix were rejected, */
/* probability T_i (1 - alpha_i), after which c_k has mean B_i.          */
/* Discontinuities (order swaps, the ellipsoid cutoff) are not           */
/* differentiated.                                                       */
/* ------------------------------------------------------------------ */

/* d alpha / d theta (11 entries) of Gaussian g for the ray (o, d). */
static void dalpha_dtheta(const orc_scene *sc, const orc_gauss *G, int64_t g, const double o[3],
                          const double d[3], double t, double alpha, double out[11])
{
    double v[3];
    for (int k = 0; k < 3; ++k) v[k] = o[k] + t * d[k] - G->mu[k];
    double Sv[3];
    for (int i = 0; i < 3; ++i)
        Sv[i] = G->Sinv[3 * i] * v[0] + G->Sinv[3 * i + 1] * v[1] + G->Sinv[3 * i + 2] * v[2];
    const double dadq = -0.5 * alpha;
    /* mean: dq/dmu = -2 Sigma^-1 v */
    for (int k = 0; k < 3; ++k) out[k] = dadq * (-2.0 * Sv[k]);
    /* rotation and scales */
    double R[9];
    quat_to_rot(sc->quats + 4 * g, R);
    double a[3], inv_s2[3];
    for (int k = 0; k < 3; ++k) {
        a[k] = R[k] * v[0] + R[3 + k] * v[1] + R[6 + k] * v[2]; /* (R^T v)_k */
        double s = exp((double)sc->log_scales[3 * g + k]);
        inv_s2[k] = 1.0 / (s * s);
        out[3 + k] = dadq * (-2.0 * a[k] * a[k] * inv_s2[k]);
    }
    /* dq/dR_jk = 2 v_j a_k / s_k^2 */
    double dR[9];
    for (int j = 0; j < 3; ++j)
        for (int k = 0; k < 3; ++k) dR[3 * j + k] = 2.0 * v[j] * a[k] * inv_s2[k];
    const float *qf = sc->quats + 4 * g;
    double qr[4] = {qf[0], qf[1], qf[2], qf[3]};
    double n = sqrt(qr[0] * qr[0] + qr[1] * qr[1] + qr[2] * qr[2] + qr[3] * qr[3]);
    double w = qr[0] / n, x = qr[1] / n, y = qr[2] / n, z = qr[3] / n;
    /* dR/dw, dR/dx, dR/dy, dR/dz of the rotation matrix of (w,x,y,z) */
    const double Dw[9] = {0, -2 * z, 2 * y, 2 * z, 0, -2 * x, -2 * y, 2 * x, 0};
    const double Dx[9] = {0, 2 * y, 2 * z, 2 * y, -4 * x, -2 * w, 2 * z, 2 * w, -4 * x};
    const double Dy[9] = {-4 * y, 2 * x, 2 * w, 2 * x, 0, 2 * z, -2 * w, 2 * z, -4 * y};
    const double Dz[9] = {-4 * z, -2 * w, 2 * x, 2 * w, -4 * z, 2 * y, 2 * x, 2 * y, 0};
    const double *D[4] = {Dw, Dx, Dy, Dz};
    double gq[4];
    for (int c = 0; c < 4; ++c) {
        double acc = 0.0;
        for (int e = 0; e < 9; ++e) acc += dR[e] * D[c][e];
        gq[c] = acc;
    }
    /* through the normalisation: (I - qhat qhat^T) / |q| */
    double qh[4] = {w, x, y, z};
    double dot = gq[0] * w + gq[1] * x + gq[2] * y + gq[3] * z;
    for (int c = 0; c < 4; ++c) out[6 + c] = dadq * (gq[c] - dot * qh[c]) / n;
    /* opacity logit */
    out[10] = alpha * (1.0 - G->opacity);
}

typedef struct {
    double *means, *log_scales, *quats, *logits, *sh;
} orc_grads;

static void add_theta(const orc_grads *gr, int64_t g, double scale, const double da[11])
{
    for (int k = 0; k < 3; ++k) {
#ifdef _OPENMP
#pragma omp atomic
#endif
        gr->means[3 * g + k] += scale * da[k];
#ifdef _OPENMP
#pragma omp atomic
#endif
        gr->log_scales[3 * g + k] += scale * da[3 + k];
    }
    for (int k = 0; k < 4; ++k) {
#ifdef _OPENMP
#pragma omp atomic
#endif
        gr->quats[4 * g + k] += scale * da[6 + k];
    }
#ifdef _OPENMP
#pragma omp atomic
#endif
    gr->logits[g] += scale * da[10];
}

/* dc/dk for the colour of Gaussian g: w_ch * mask_ch * Y_K, accumulated. */
static void add_sh(const orc_scene *sc, const orc_grads *gr, int64_t g, const double *Y,
                   const double rgb_raw_pos[3], const double w[3])
{
    int K = (sc->sh_degree + 1) * (sc->sh_degree + 1);
    for (int ch = 0; ch < 3; ++ch) {
        if (!(rgb_raw_pos[ch] > 0.0)) continue; /* max(0, .) clamp */
        for (int i = 0; i < K; ++i) {
            double b = i == 0 ? 1.0 : Y[i];
#ifdef _OPENMP
#pragma omp atomic
#endif
            gr->sh[((size_t)g * K + i) * 3 + ch] += w[ch] * b;
        }
    }
}

/* Raw (unclamped) colour, to know which channels pass the clamp. */
static void sh_raw(const orc_scene *sc, int64_t g, const double *Y, double raw[3])
{
    int K = (sc->sh_degree + 1) * (sc->sh_degree + 1);
    const float *k = sc->sh + (size_t)g * K * 3;
    for (int ch = 0; ch < 3; ++ch) {
        double acc = (double)k[ch];
        for (int i = 1; i < K; ++i) acc += Y[i] * (double)k[3 * i + ch];
        raw[ch] = acc;
    }
}

/* Exported: gradients of G = sum_p d_rgb[p] . L_p over the listed pixels.
 * mode 0: exact blend (Eq. 3). mode 1: the stochastic estimator averaged
 * over the spp * n_hits samples of each pixel, same draws as rendering.
 * Gradient arrays (FP64, caller-zeroed, same layouts as the parameters)
 * are accumulated. Returns the number of threads used. */
int orc_grad_pinhole(const orc_scene *sc, const orc_pinhole *cam, const orc_params *p,
                     int64_t n_pix, const int64_t *pix, const double *d_rgb, int mode,
                     double *g_means, double *g_log_scales, double *g_quats, double *g_logits,
                     double *g_sh, int n_threads)
{
    orc_gauss *act = activate_all(sc);
    orc_grads gr = {g_means, g_log_scales, g_quats, g_logits, g_sh};
    int64_t S = (int64_t)p->spp * p->n_hits;
    int used = 1;
#ifdef _OPENMP
    if (n_threads <= 0) n_threads = omp_get_max_threads();
#pragma omp parallel num_threads(n_threads)
#endif
    {
#ifdef _OPENMP
#pragma omp single
        used = omp_get_num_threads();
#endif
        cand_list L = {0, 0, 0};
        double *suffix = NULL;
        int64_t suffix_cap = 0;
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 2)
#endif
        for (int64_t r = 0; r < n_pix; ++r) {
            int32_t x = (int32_t)(pix[r] % cam->width), y = (int32_t)(pix[r] / cam->width);
            double o[3], d[3];
            uint32_t rid;
            orc_camera_ray(cam, x, y, o, d, &rid);
            collect(sc, act, o, d, p->t_min, p->t_max, &L);
            qsort(L.v, (size_t)L.n, sizeof(orc_cand), cand_cmp);
            double Y[16];
            orc_sh_basis(sc->sh_degree, d, Y);
            const double *g = d_rgb + 3 * r;
            if (mode == 0) {
                if (L.n + 1 > suffix_cap) {
                    suffix_cap = 2 * (L.n + 1);
                    suffix = (double *)realloc(suffix, (size_t)suffix_cap * 3 * sizeof(double));
                }
                /* suffix[i] = blend of candidates i.. plus background */
                for (int ch = 0; ch < 3; ++ch) suffix[3 * L.n + ch] = p->bg[ch];
                for (int64_t i = L.n - 1; i >= 0; --i)
                    for (int ch = 0; ch < 3; ++ch)
                        suffix[3 * i + ch] = L.v[i].alpha * L.v[i].rgb[ch] +
                                             (1.0 - L.v[i].alpha) * suffix[3 * (i + 1) + ch];
                double T = 1.0;
                for (int64_t i = 0; i < L.n; ++i) {
                    const orc_cand *c = &L.v[i];
                    double dG = 0.0;
                    for (int ch = 0; ch < 3; ++ch)
                        dG += g[ch] * (c->rgb[ch] - suffix[3 * (i + 1) + ch]);
                    dG *= T;
                    double da[11];
                    dalpha_dtheta(sc, &act[c->gid], c->gid, o, d, c->t, c->alpha, da);
                    add_theta(&gr, c->gid, dG, da);
                    double raw[3], w[3];
                    sh_raw(sc, c->gid, Y, raw);
                    for (int ch = 0; ch < 3; ++ch) w[ch] = T * c->alpha * g[ch];
                    add_sh(sc, &gr, c->gid, Y, raw, w);
                    T *= (1.0 - c->alpha);
                }
            } else {
                for (int64_t s = 0; s < S; ++s) {
                    int64_t win = -1;
                    for (int64_t i = 0; i < L.n; ++i) {
                        double xi = orc_xi(p->seed, rid, (uint32_t)L.v[i].gid, (uint32_t)s,
                                           p->stream_tag);
                        if (xi < L.v[i].alpha) { win = i; break; } /* sorted: first accepted */
                    }
                    const double *ck = win >= 0 ? L.v[win].rgb : p->bg;
                    if (win >= 0) {
                        double raw[3], w[3];
                        sh_raw(sc, L.v[win].gid, Y, raw);
                        for (int ch = 0; ch < 3; ++ch) w[ch] = g[ch] / (double)S;
                        add_sh(sc, &gr, L.v[win].gid, Y, raw, w);
                    }
                    int64_t n_front = win >= 0 ? win : L.n;
                    for (int64_t i = 0; i < n_front; ++i) {
                        const orc_cand *c = &L.v[i];
                        double dG = 0.0;
                        for (int ch = 0; ch < 3; ++ch) dG += g[ch] * (c->rgb[ch] - ck[ch]);
                        dG /= (double)S * (1.0 - c->alpha);
                        double da[11];
                        dalpha_dtheta(sc, &act[c->gid], c->gid, o, d, c->t, c->alpha, da);
                        add_theta(&gr, c->gid, dG, da);
                    }
                }
            }
        }
        free(L.v);
        free(suffix);
    }
    free(act);
    return used;
}

/* ------------------------------------------------------------------ */
/* Scenes with a ground quad, point lights and one diffuse bounce (the  */
/* Monte Carlo path-tracing integration of Sec. 5). Gaussians are        */
/* emissive; the ground is Lambertian. Per sample s of a pixel:          */
/*   camera ray -> closest accepted Gaussian (t_g) or ground (t_q),       */
/*   the nearer one shades (ground on ties);                              */
/*   ground: albedo/pi sum_l I_l V_l cos_l / r_l^2 + albedo L_b,          */
/*   V_l = no accepted Gaussian on the shadow segment (tag 1 + l),        */
/*   L_b = colour of the closest accepted Gaussian along a cosine-        */
/*   weighted bounce direction (tag 9), else the background.              */
/* Secondary rays are float32 values from fixed sequences of correctly    */
/* rounded float operations; Gaussian evaluations are FP64.              */
/* ------------------------------------------------------------------ */
typedef struct {
    float position[3];
    float intensity[3];
} orc_light;

typedef struct {
    int32_t n_lights;
    orc_light lights[8];
    int32_t has_ground;
    float ground_y;
    float ground_half_extent;
    float ground_albedo[3];
    int32_t bounce;
    float shadow_eps;
} orc_extras;

/* Closest (or, with any_hit, some) accepted Gaussian on a float32 ray with
 * range (t_min, t_max); returns its id or -1, *t_out its depth. */
static int64_t accepted_on_ray(const orc_scene *sc, const orc_gauss *act, const float of[3],
                               const float df[3], double t_min, double t_max, uint64_t seed,
                               uint32_t ray_id, uint32_t s, uint32_t tag, int any_hit,
                               double *t_out)
{
    double o[3] = {of[0], of[1], of[2]}, d[3] = {df[0], df[1], df[2]};
    int64_t win = -1;
    double tw = INFINITY;
    for (int64_t g = 0; g < sc->M; ++g) {
        double t, q;
        gauss1d(&act[g], o, d, &t, &q);
        if (!(t > t_min && t < t_max)) continue;
        if (!(q <= ORC_S2)) continue;
        double alpha = act[g].opacity * exp(-0.5 * q);
        if (!(orc_xi(seed, ray_id, (uint32_t)g, s, tag) < alpha)) continue;
        if (win < 0 || lex_less(t, (int32_t)g, tw, (int32_t)win)) {
            win = g;
            tw = t;
            if (any_hit) break;
        }
    }
    if (t_out) *t_out = tw;
    return win;
}

static void colour_of(const orc_scene *sc, int64_t g, const float df[3], double rgb[3])
{
    double d[3] = {df[0], df[1], df[2]};
    double Y[16];
    orc_sh_basis(sc->sh_degree, d, Y);
    sh_colour(sc, g, Y, rgb);
}

/* Cosine-weighted bounce direction about +y from Philox draws (exported
 * for tests). */
void orc_bounce_dir(uint64_t seed, uint32_t ray_id, uint32_t s, float d[3])
{
    uint32_t key[2] = {(uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32)};
    float u[3] = {0.0f, 1.0f, 0.0f};
    for (uint32_t attempt = 0; attempt < 16; ++attempt) {
        uint32_t ctr[4] = {ray_id, attempt, s, 16u}, w[4];
        orc_philox4x32_10(ctr, key, w);
        float v[3];
        for (int i = 0; i < 3; ++i) {
            float f = (float)(w[i] >> 8) * (1.0f / 16777216.0f);
            v[i] = 2.0f * f - 1.0f;
        }
        float r2 = v[0] * v[0];
        r2 = r2 + v[1] * v[1];
        r2 = r2 + v[2] * v[2];
        if (r2 > 1e-8f && r2 <= 1.0f) {
            float n = sqrtf(r2);
            for (int i = 0; i < 3; ++i) u[i] = v[i] / n;
            break;
        }
    }
    float b[3] = {u[0], 1.0f + u[1], u[2]};
    float n2 = b[0] * b[0];
    n2 = n2 + b[1] * b[1];
    n2 = n2 + b[2] * b[2];
    if (!(n2 > 1e-12f)) {
        d[0] = 0.0f; d[1] = 1.0f; d[2] = 0.0f;
        return;
    }
    float n = sqrtf(n2);
    for (int i = 0; i < 3; ++i) d[i] = b[i] / n;
}

/* Ground point of a float32 camera ray (o, d): tq = (ground_y - o.y) / d.y,
 * p = o + tq d with p.y = ground_y, each operation rounded once in float32.
 * Returns 1 when the ray meets the quad inside its range, else 0 (tq is
 * then +inf). */
static int ground_point(const orc_extras *ex, const float o[3], const float d[3], double t_min,
                        float *tq_out, float gp[3])
{
    int ground = 0;
    float tq = INFINITY;
    gp[0] = gp[1] = gp[2] = 0.0f;
    if (ex && ex->has_ground && d[1] != 0.0f) {
        tq = (ex->ground_y - o[1]) / d[1];
        float ax = tq * d[0], az = tq * d[2];
        gp[0] = o[0] + ax;
        gp[1] = ex->ground_y;
        gp[2] = o[2] + az;
        ground = (double)tq > t_min && fabsf(gp[0]) <= ex->ground_half_extent &&
                 fabsf(gp[2]) <= ex->ground_half_extent;
        if (!ground) tq = INFINITY;
    }
    *tq_out = tq;
    return ground;
}

/* Shadow ray from ground point gp to light l in float32: unit direction om,
 * distance dist and its square. Returns 0 when the light is not above the
 * ground (no contribution). */
static int light_ray(const orc_extras *ex, int l, const float gp[3], float om[3], float *dist_out,
                     float *dist2_out)
{
    float w[3];
    for (int i = 0; i < 3; ++i) w[i] = ex->lights[l].position[i] - gp[i];
    float dist2 = w[0] * w[0];
    dist2 = dist2 + w[1] * w[1];
    dist2 = dist2 + w[2] * w[2];
    float dist = sqrtf(dist2);
    for (int i = 0; i < 3; ++i) om[i] = w[i] / dist;
    *dist_out = dist;
    *dist2_out = dist2;
    return om[1] > 0.0f && dist2 > 0.0f;
}

/* Exported for the tests' mismatch classifier: the float32 rays of sample s
 * of pixel (x, y) of a camera in the scene renderer. out[46]:
 *   [0..2] camera origin, [3..5] camera direction, [6] ray id (its bits),
 *   [7] ground tq (+inf when the quad is missed), [8..10] ground point,
 *   [11..13] bounce direction, and per light l < 8: [14 + 4l .. 16 + 4l]
 *   the shadow ray's direction, [17 + 4l] its length, or -1 when light l
 *   does not contribute. Returns 1 when the camera ray meets the ground. */
int orc_scene_sample_rays(const orc_pinhole *cam, const orc_extras *ex, const orc_params *p,
                          int32_t x, int32_t y, uint32_t s, float *out)
{
    double od[3], dd[3];
    uint32_t rid;
    orc_camera_ray(cam, x, y, od, dd, &rid);
    float o[3] = {(float)od[0], (float)od[1], (float)od[2]};
    float d[3] = {(float)dd[0], (float)dd[1], (float)dd[2]};
    for (int i = 0; i < 3; ++i) {
        out[i] = o[i];
        out[3 + i] = d[i];
    }
    memcpy(&out[6], &rid, sizeof(rid));
    float tq, gp[3];
    int ground = ground_point(ex, o, d, p->t_min, &tq, gp);
    out[7] = tq;
    for (int i = 0; i < 3; ++i) out[8 + i] = gp[i];
    float db[3];
    orc_bounce_dir(p->seed, rid, s, db);
    for (int i = 0; i < 3; ++i) out[11 + i] = db[i];
    for (int l = 0; l < 8; ++l) {
        float om[3] = {0.0f, 0.0f, 0.0f}, dist = -1.0f, dist2 = 0.0f;
        int ok = ground && ex && l < ex->n_lights && light_ray(ex, l, gp, om, &dist, &dist2);
        for (int i = 0; i < 3; ++i) out[14 + 4 * l + i] = om[i];
        out[14 + 4 * l + 3] = ok ? dist : -1.0f;
    }
    return ground;
}

/* Exported: render items (view[i], pix[i]) of the given cameras.
 * est [n][3]; diag [n][spp][3] = {camera hit (id, -2 ground, -1 none),
 * bounce hit (id or -1), visible-light bits} (nullable). */
int orc_render_scene(const orc_scene *sc, const orc_pinhole *cams, int32_t n_views,
                     const orc_extras *ex, const orc_params *p, int64_t n_items,
                     const int32_t *view, const int64_t *pix, double *est, int32_t *diag,
                     int n_threads)
{
    (void)n_views;
    orc_gauss *act = activate_all(sc);
    const int32_t S = p->spp;
    int used = 1;
#ifdef _OPENMP
    if (n_threads <= 0) n_threads = omp_get_max_threads();
#pragma omp parallel for schedule(dynamic, 1) num_threads(n_threads)
#endif
    for (int64_t it = 0; it < n_items; ++it) {
#ifdef _OPENMP
        if (it == 0) used = omp_get_num_threads();
#endif
        const orc_pinhole *cam = &cams[view[it]];
        int32_t x = (int32_t)(pix[it] % cam->width), y = (int32_t)(pix[it] / cam->width);
        double od[3], dd[3];
        uint32_t rid;
        orc_camera_ray(cam, x, y, od, dd, &rid);
        float o[3] = {(float)od[0], (float)od[1], (float)od[2]};
        float d[3] = {(float)dd[0], (float)dd[1], (float)dd[2]};
        /* ground point in float32 */
        float tq, gp[3];
        int ground = ground_point(ex, o, d, p->t_min, &tq, gp);
        double acc[3] = {0.0, 0.0, 0.0};
        for (int32_t s = 0; s < S; ++s) {
            double tg;
            int64_t g = accepted_on_ray(sc, act, o, d, p->t_min, p->t_max, p->seed, rid,
                                        (uint32_t)s, p->stream_tag, 0, &tg);
            double c[3] = {p->bg[0], p->bg[1], p->bg[2]};
            int32_t dcam = -1, dbounce = -1, dvis = 0;
            int gauss = g >= 0 && tg < (double)tq;
            int on_ground = ground && !gauss;
            if (gauss) {
                colour_of(sc, g, d, c);
                dcam = (int32_t)g;
            }
            if (on_ground) {
                c[0] = c[1] = c[2] = 0.0;
                dcam = -2;
                for (int l = 0; l < ex->n_lights; ++l) {
                    float om[3], dist, dist2;
                    if (!light_ray(ex, l, gp, om, &dist, &dist2)) continue;
                    int64_t blocker = accepted_on_ray(sc, act, gp, om, ex->shadow_eps, dist, p->seed,
                                                      rid, (uint32_t)s, 1u + (uint32_t)l, 1, NULL);
                    if (blocker >= 0) continue;
                    dvis |= 1 << l;
                    for (int ch = 0; ch < 3; ++ch)
                        c[ch] += (double)ex->ground_albedo[ch] / M_PI *
                                 (double)ex->lights[l].intensity[ch] * (double)om[1] /
                                 (double)dist2;
                }
                if (ex->bounce) {
                    float db[3];
                    orc_bounce_dir(p->seed, rid, (uint32_t)s, db);
                    int64_t gb = accepted_on_ray(sc, act, gp, db, ex->shadow_eps, INFINITY, p->seed,
                                                 rid, (uint32_t)s, 9u, 0, NULL);
                    double lb[3] = {p->bg[0], p->bg[1], p->bg[2]};
                    if (gb >= 0) {
                        colour_of(sc, gb, db, lb);
                        dbounce = (int32_t)gb;
                    }
                    for (int ch = 0; ch < 3; ++ch) c[ch] += (double)ex->ground_albedo[ch] * lb[ch];
                }
            }
            for (int ch = 0; ch < 3; ++ch) acc[ch] += c[ch];
            if (diag) {
                int32_t *dg = diag + ((size_t)it * S + (size_t)s) * 3;
                dg[0] = dcam;
                dg[1] = dbounce;
                dg[2] = dvis;
            }
        }
        if (est)
            for (int ch = 0; ch < 3; ++ch) est[3 * it + ch] = acc[ch] / (double)S;
    }
    free(act);
    return used;
}
