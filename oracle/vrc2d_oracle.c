/*
 * vrc2d_oracle.c -- plain FP64 CPU oracle for the paper's two-dimensional world
 * (Marco, Jarabo, Jarosz, Gutierrez, TOG 37(2) 2018, Sec. 3 "2D and 3D Light
 * Transport in Participating Media", Sec. 4 in 2D, App. A, App. B, Eq. radiusAniso2D).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the benchmark's
 * CPU-baseline leg may load this library.  It shares no code with the CUDA library.
 *
 * The 2D world is the intrinsic planar model of Sec. 3: light travels, scatters and
 * is absorbed within the plane; radiance from a point source falls off as 1/r; phase
 * functions are normalised over the circle.  Geometry is a set of line segments
 * ("curves") in the unit square, which the homogeneous medium fills.
 *
 * Readings this file fixes (2D counterparts of the 3D readings, numbered D1..D9):
 *  D1  the cached quantity is L = int f L_i dtheta over the circle, f = 1/(2 pi)
 *      (isotropic medium, the paper's restriction; Sec. 3 normalises over the circle).
 *  D2  ray set: N equal-angle strata theta_j = 2 pi (j + u_j) / N, one jittered ray
 *      each (Sec. 6 "Implementation", 2D case), u_j = splitmix64 jitter with band 0,
 *      bin j and stream 2.
 *  D3  cells are the segments between angularly adjacent vertices (j, j + 1 mod N) of
 *      a shell; the cell radiance is L_j = f T L_o theta_j with theta_j the angle the
 *      cell subtends (App. B's F = theta / 2 pi times 2 pi, the 2D counterpart of R2).
 *  D4  theta_j is App. B's arccos of the normalised dot product, signed by the cross
 *      product of (y_0 - x, y_1 - x) so that a closed shell sums to 2 pi (the 2D
 *      counterpart of R5); its gradient and Hessian are App. B's expressions times
 *      that sign.
 *  D5  shells, clamping, furthest point, tie averaging and escaped rays as in 3D
 *      (R7, R9, R10): t_k = (k - 1/2) dt, vertices beyond the hit sit at the hit with
 *      zero radiance, the furthest endpoint freezes T and L_o, exact ties average.
 *  D6  vertex radiance: two-sided Lambertian curves, f_r = rho / 2 (normalised over
 *      the half circle), irradiance I |cos| T V / d from a point light; medium vertices
 *      single-scatter, L_o = f I T V / d.  Shadow rays start 1e-5 along the normal
 *      facing x.  grad L_o = 0.
 *  D7  surface shell weight 1, medium shells sigma_s dt (1 / pdf, Sec. 4).
 *  D8  radius from the 2x2 luminance Hessian: Eq. radiusAniso2D,
 *      R = (4 L_Y eps / (pi max|lambda|))^(1/4), clamps as R15.
 *  D9  ray hits: smallest t, then lowest segment id; t_min = 1e-6.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define O2_PI 3.14159265358979323846
#define O2_TMIN 1e-6
#define O2_SHADOW_OFFSET 1e-5
#define O2_NEAR 1e-5   /* near-tie margin (scene units) of a discrete decision */

enum { ST_NONFINITE = 1, ST_CLAMP_LO = 2, ST_CLAMP_HI = 4 };

typedef struct {
    int n_segs;
    const float* seg;        /* [n][4]: x0 y0 x1 y1 */
    const float* albedo;     /* [n][3] */
    float sigma_s, sigma_a;
    int n_lights;
    const float* light_pos;  /* [n][2] */
    const float* light_I;    /* [n][3] */
    int circle_mode;         /* 1: analytic circle of constant outgoing radiance, no segments */
    float circle_c[2], circle_r, circle_Le[3];
} o2_scene;

typedef struct {
    int n_dirs;
    float dt, eps;
    uint64_t seed;
    float r_min, r_max;
    int64_t rec_base;
} o2_params;

typedef struct { double x, y; } v2;
static v2 mk2(double x, double y) { v2 r = {x, y}; return r; }
static v2 sub2(v2 a, v2 b) { return mk2(a.x - b.x, a.y - b.y); }
static v2 add2(v2 a, v2 b) { return mk2(a.x + b.x, a.y + b.y); }
static v2 scl2(v2 a, double s) { return mk2(a.x * s, a.y * s); }
static double dot2(v2 a, v2 b) { return a.x * b.x + a.y * b.y; }
static double crs2(v2 a, v2 b) { return a.x * b.y - a.y * b.x; }
static double nrm2(v2 a) { return sqrt(dot2(a, a)); }

/* value, gradient (2) and Hessian (xx, xy, yy) of a scalar function of x */
typedef struct { double v, g[2], h[3]; } s2fun;

/* ------------------------------------------------------------- jitter (D2) */
static uint64_t splitmix64(uint64_t x) {
    uint64_t z = x + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
static double jitter2(uint64_t seed, int64_t rec, int j) {
    uint64_t key = seed ^ ((uint64_t)rec << 32) ^ (uint64_t)j ^ (2ull << 60);
    return (double)(splitmix64(key) >> 40) * (1.0 / 16777216.0);
}
static v2 ray_dir2(const o2_params* p, int64_t rec, int j) {
    double th = 2.0 * O2_PI * ((double)j + jitter2(p->seed, rec, j)) / (double)p->n_dirs;
    return mk2(cos(th), sin(th));
}

/* ---------------------------------------------------------- ray casting (D9) */
static v2 seg_a(const o2_scene* s, int i) { return mk2(s->seg[4 * i], s->seg[4 * i + 1]); }
static v2 seg_b(const o2_scene* s, int i) { return mk2(s->seg[4 * i + 2], s->seg[4 * i + 3]); }

/* x + t d = a + u (b - a); returns 1 with t and the distance of the hit from the nearer
 * endpoint (scene units) */
static int hit_seg(v2 x, v2 d, v2 a, v2 b, double* t, double* edge) {
    v2 e = sub2(b, a), w = sub2(a, x);
    double den = crs2(d, e);
    if (den == 0.0) return 0;
    double tt = crs2(w, e) / den;
    double u = crs2(w, d) / den;
    if (!(tt > O2_TMIN) || u < 0.0 || u > 1.0) return 0;
    *t = tt;
    *edge = fmin(u, 1.0 - u) * nrm2(e);
    return 1;
}

/* closest hit: segment id or -1; *near_edge = smallest endpoint distance among the hit
 * and any segment whose endpoint the ray passes within O2_NEAR of before the hit */
static int closest2(const o2_scene* s, v2 x, v2 d, double* t_out, double* near_edge) {
    int best = -1;
    double bt = 1e300, be = 1e300;
    for (int i = 0; i < s->n_segs; ++i) {
        double t, e;
        if (hit_seg(x, d, seg_a(s, i), seg_b(s, i), &t, &e) && t < bt) { bt = t; best = i; be = e; }
    }
    double ne = best >= 0 ? be : 1e300;
    for (int i = 0; i < s->n_segs; ++i) {   /* endpoints grazed before the hit */
        v2 ends[2] = {seg_a(s, i), seg_b(s, i)};
        for (int q = 0; q < 2; ++q) {
            v2 w = sub2(ends[q], x);
            double tp = dot2(w, d);
            if (tp <= O2_TMIN || tp > bt) continue;
            double dist = fabs(crs2(d, w));
            if (dist < ne) ne = dist;
        }
    }
    *t_out = bt;
    if (near_edge) *near_edge = ne;
    return best;
}

static int occluded2(const o2_scene* s, v2 o, v2 d, double limit, double* near_edge) {
    double ne = 1e300;
    int occ = 0;
    for (int i = 0; i < s->n_segs; ++i) {
        double t, e;
        if (hit_seg(o, d, seg_a(s, i), seg_b(s, i), &t, &e) && t < limit) {
            occ = 1;
            if (e < ne) ne = e;
        }
        v2 ends[2] = {seg_a(s, i), seg_b(s, i)};
        for (int q = 0; q < 2; ++q) {
            v2 w = sub2(ends[q], o);
            double tp = dot2(w, d);
            if (tp <= O2_TMIN || tp >= limit) continue;
            double dist = fabs(crs2(d, w));
            if (dist < ne) ne = dist;
        }
    }
    if (near_edge) *near_edge = ne;
    return occ;
}

static double square_exit(v2 x, v2 d) {
    double t = 1e300;
    double c[2] = {x.x, x.y}, dd[2] = {d.x, d.y};
    for (int a = 0; a < 2; ++a) {
        if (dd[a] > 0) t = fmin(t, (1.0 - c[a]) / dd[a]);
        else if (dd[a] < 0) t = fmin(t, (0.0 - c[a]) / dd[a]);
    }
    return t;
}

/* circle mode: distance from x (inside) to the circle along d */
static double circle_exit(const o2_scene* s, v2 x, v2 d) {
    v2 w = sub2(x, mk2(s->circle_c[0], s->circle_c[1]));
    double b = dot2(w, d), c = dot2(w, w) - (double)s->circle_r * s->circle_r;
    return -b + sqrt(b * b - c);
}

/* ------------------------------------------------------ vertex radiance (D6) */
/* Each light adds its term unless a segment blocks the shadow ray.  dLo[c] collects the
 * terms whose visibility decision lies within O2_NEAR of flipping (the ray passes that
 * close to a segment endpoint): the most a float-precision evaluation may differ by. */
static void light_terms(const o2_scene* s, v2 o, v2 n_side, int surface, double albedo_scale, const float* albedo,
                        double Lo[3], double dLo[3]) {
    double sig_t = (double)s->sigma_s + (double)s->sigma_a;
    for (int L = 0; L < s->n_lights; ++L) {
        v2 l = mk2(s->light_pos[2 * L], s->light_pos[2 * L + 1]);
        v2 tl = sub2(l, o);
        double dist = nrm2(tl);
        v2 ld = scl2(tl, 1.0 / dist);
        double cs = 1.0;
        if (surface) {
            cs = dot2(n_side, ld);
            if (cs <= 0) continue;                      /* light behind the lit side */
        }
        double ne;
        int occ = occluded2(s, o, ld, dist, &ne);
        double T = exp(-sig_t * dist);
        for (int c = 0; c < 3; ++c) {
            double a = surface ? albedo_scale * (double)albedo[c] : albedo_scale;
            double term = a * (double)s->light_I[3 * L + c] * cs * T / dist;
            if (!occ) Lo[c] += term;
            if (ne < O2_NEAR) dLo[c] += fabs(term);
        }
    }
}

static void surface_Lo(const o2_scene* s, int id, v2 y, v2 d, double Lo[3], double dLo[3]) {
    Lo[0] = Lo[1] = Lo[2] = 0.0;
    v2 a = seg_a(s, id), b = seg_b(s, id);
    v2 e = sub2(b, a);
    v2 n = scl2(mk2(-e.y, e.x), 1.0 / nrm2(e));
    if (dot2(n, d) > 0) n = scl2(n, -1.0);          /* normal facing x (d points away from x) */
    light_terms(s, add2(y, scl2(n, O2_SHADOW_OFFSET)), n, 1, 0.5, &s->albedo[3 * id], Lo, dLo);
}

static void medium_Lo(const o2_scene* s, v2 y, double Lo[3], double dLo[3]) {
    Lo[0] = Lo[1] = Lo[2] = 0.0;
    light_terms(s, y, mk2(0, 0), 0, 1.0 / (2.0 * O2_PI), NULL, Lo, dLo);
}

/* ------------------------------------------------- transmittance (App. A) */
static void transmittance2(v2 x, v2 y, double sigma_t, s2fun* T) {
    v2 w = sub2(x, y);                 /* the paper's yx: from y to x */
    double r = nrm2(w);
    double Tv = exp(-sigma_t * r);
    T->v = Tv;
    T->g[0] = -sigma_t * w.x / r * Tv;
    T->g[1] = -sigma_t * w.y / r * Tv;
    double a = 1.0 / r, b = 1.0 / (r * r * r), c = sigma_t / (r * r);
    T->h[0] = -sigma_t * (a - b * w.x * w.x - c * w.x * w.x) * Tv;
    T->h[1] = -sigma_t * (-b * w.x * w.y - c * w.x * w.y) * Tv;
    T->h[2] = -sigma_t * (a - b * w.y * w.y - c * w.y * w.y) * Tv;
}

/* --------------------------------------- segment form factor (App. B, D4) */
/* theta = sign(cross) * arccos(c), c = (y0 - x).(y1 - x) / (r0 r1), with App. B's
 * gradient and Hessian of arccos(c) (times 2 pi: the angle itself, D3).  Returns 0
 * for a degenerate cell (collinear with x or an endpoint at x). */
static int segment_angle(v2 x, v2 y0, v2 y1, s2fun* F) {
    v2 u = sub2(y0, x), v = sub2(y1, x);       /* the paper's xy_0, xy_1 */
    double r0 = nrm2(u), r1 = nrm2(v);
    double A = crs2(u, v);
    memset(F, 0, sizeof(*F));
    if (r0 == 0.0 || r1 == 0.0 || A == 0.0) return 0;
    double sg = A > 0 ? 1.0 : -1.0;
    double c = dot2(u, v) / (r0 * r1);
    if (c > 1.0) c = 1.0;
    if (c < -1.0) c = -1.0;
    double s2 = 1.0 - c * c;
    if (!(s2 > 0.0)) return 0;
    double sq = sqrt(s2);
    /* grad c = c u / r0^2 + c v / r1^2 - (u + v) / (r0 r1) */
    double gc[2] = {c * u.x / (r0 * r0) + c * v.x / (r1 * r1) - (u.x + v.x) / (r0 * r1),
                    c * u.y / (r0 * r0) + c * v.y / (r1 * r1) - (u.y + v.y) / (r0 * r1)};
    /* J(grad c) from App. B: J(xy_i) = -I */
    double J[2][2];
    const double uu[2] = {u.x, u.y}, vv[2] = {v.x, v.y};
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 2; ++j) {
            double I = i == j ? 1.0 : 0.0;
            /* J(xy_0 / (r0 r1)) and J(xy_1 / (r0 r1)) */
            double J0 = -I / (r0 * r1) + uu[i] * uu[j] / (r0 * r0 * r0 * r1) + uu[i] * vv[j] / (r0 * r1 * r1 * r1);
            double J1 = -I / (r0 * r1) + vv[i] * uu[j] / (r0 * r0 * r0 * r1) + vv[i] * vv[j] / (r0 * r1 * r1 * r1);
            /* J(c xy_i / r_i^2) */
            double K0 = -c * I / (r0 * r0) + uu[i] * gc[j] / (r0 * r0) + 2.0 * c * uu[i] * uu[j] / (r0 * r0 * r0 * r0);
            double K1 = -c * I / (r1 * r1) + vv[i] * gc[j] / (r1 * r1) + 2.0 * c * vv[i] * vv[j] / (r1 * r1 * r1 * r1);
            J[i][j] = -J0 - J1 + K0 + K1;
        }
    F->v = sg * acos(c);
    F->g[0] = -sg * gc[0] / sq;
    F->g[1] = -sg * gc[1] / sq;
    double k = c / (s2 * sq);
    /* symmetrise the Jacobian (the exact one is symmetric; rounding is not) */
    F->h[0] = -sg * (J[0][0] / sq + k * gc[0] * gc[0]);
    F->h[1] = -sg * (0.5 * (J[0][1] + J[1][0]) / sq + k * gc[0] * gc[1]);
    F->h[2] = -sg * (J[1][1] / sq + k * gc[1] * gc[1]);
    return 1;
}

/* -------------------------------------------------------- one record (Sec. 4) */
/* out layout (doubles): L[3], L_ss[3], L_ms[3], grad[3][2], grad_ss[3][2], grad_ms[3][2],
 * hess[3][3] (xx xy yy), hess_ss, hess_ms, L_ff[3], radius, eig[2], status, n_shells,
 * primary near-tie count, budgets of L, grad and hess per channel (the change that
 * flipping the near-tie shadow and clamp decisions could make) */
enum {
    O_L = 0, O_LSS = 3, O_LMS = 6, O_G = 9, O_GSS = 15, O_GMS = 21, O_H = 27, O_HSS = 36, O_HMS = 45,
    O_LFF = 54, O_R = 57, O_EIG = 58, O_ST = 60, O_K = 61, O_PNEAR = 62, O_BL = 63, O_BG = 66, O_BH = 69,
    O2_STRIDE = 72
};

static const double LUM2[3] = {0.2126, 0.7152, 0.0722};

/* Eq. radiusAniso2D with the largest |eigenvalue| of the 2x2 luminance Hessian (D8) */
double o2_radius(double LY, const double* h3, double eps, double r_min, double r_max, int* status, double* lam) {
    double a = h3[0], b = h3[1], c = h3[2];
    double m = 0.5 * (a + c), dlt = sqrt(0.25 * (a - c) * (a - c) + b * b);
    lam[0] = m - dlt;
    lam[1] = m + dlt;
    double lmax = fmax(fabs(lam[0]), fabs(lam[1]));
    if (!isfinite(LY) || !isfinite(lmax)) { *status |= ST_NONFINITE | ST_CLAMP_LO; return r_min; }
    if (!(LY > 0)) { *status |= ST_CLAMP_LO; return r_min; }
    if (lmax == 0.0) { *status |= ST_CLAMP_HI; return r_max; }
    double R = pow(4.0 * LY * eps / (O2_PI * lmax), 0.25);
    if (R < r_min) { *status |= ST_CLAMP_LO; return r_min; }
    if (R > r_max) { *status |= ST_CLAMP_HI; return r_max; }
    return R;
}

typedef struct {
    double L[3], g[6], h[9];        /* cell sums of one part */
    double bL[3], bg[3], bh[3];     /* budgets */
} acc2;

/* Cell (y[0], y[1]) of a shell: the furthest endpoint(s) freeze T and L_o (mean over
 * exact ties, D5); L_j = f T L_o theta and its derivatives by the product rule.  unc[q]
 * marks an endpoint whose radiance (dLo) or clamp decision (clamp_unc) is uncertain. */
static void cell2(v2 x, const v2 y[2], const double t[2], const double* Lo[2], const double* dLo[2],
                  const int clamp_unc[2], double sigma_t, double w, acc2* A, int* degen) {
    s2fun F;
    if (!segment_angle(x, y[0], y[1], &F)) { ++*degen; return; }
    double tmax = fmax(t[0], t[1]);
    int far[2], nf = 0;
    for (int q = 0; q < 2; ++q)
        if (t[q] == tmax) far[nf++] = q;
    s2fun T[2];
    for (int q = 0; q < 2; ++q) transmittance2(x, y[q], sigma_t, &T[q]);
    const double f = 1.0 / (2.0 * O2_PI);
    int any_clamp = clamp_unc[0] || clamp_unc[1];
    for (int c = 0; c < 3; ++c) {
        double Lr = 0, gr[2] = {0, 0}, hr[3] = {0, 0, 0};
        double ub = 0;                      /* bound on |change of L_o T| */
        for (int k = 0; k < nf; ++k) {
            int q = far[k];
            double lo = Lo[q][c] / nf;
            Lr += lo * T[q].v;
            for (int e = 0; e < 2; ++e) gr[e] += lo * T[q].g[e];
            for (int e = 0; e < 3; ++e) hr[e] += lo * T[q].h[e];
            ub += dLo[q][c] / nf;
        }
        if (any_clamp)                      /* the furthest set may change: any endpoint */
            for (int q = 0; q < 2; ++q) ub += fabs(Lo[q][c]) + dLo[q][c];
        A->L[c] += w * f * Lr * F.v;
        A->g[2 * c + 0] += w * f * (gr[0] * F.v + Lr * F.g[0]);
        A->g[2 * c + 1] += w * f * (gr[1] * F.v + Lr * F.g[1]);
        A->h[3 * c + 0] += w * f * (hr[0] * F.v + 2.0 * gr[0] * F.g[0] + Lr * F.h[0]);
        A->h[3 * c + 1] += w * f * (hr[1] * F.v + gr[0] * F.g[1] + gr[1] * F.g[0] + Lr * F.h[1]);
        A->h[3 * c + 2] += w * f * (hr[2] * F.v + 2.0 * gr[1] * F.g[1] + Lr * F.h[2]);
        if (ub > 0) {
            /* |d(T theta)| with T at the larger of the endpoints' transmittances */
            double Tm = fmax(T[0].v, T[1].v);
            double gT = fmax(hypot(T[0].g[0], T[0].g[1]), hypot(T[1].g[0], T[1].g[1]));
            double hT = fmax(fabs(T[0].h[0]) + 2 * fabs(T[0].h[1]) + fabs(T[0].h[2]),
                             fabs(T[1].h[0]) + 2 * fabs(T[1].h[1]) + fabs(T[1].h[2]));
            double gF = hypot(F.g[0], F.g[1]), hF = fabs(F.h[0]) + 2 * fabs(F.h[1]) + fabs(F.h[2]);
            A->bL[c] += w * f * ub * Tm * fabs(F.v);
            A->bg[c] += w * f * ub * (gT * fabs(F.v) + Tm * gF);
            A->bh[c] += w * f * ub * (hT * fabs(F.v) + 2 * gT * gF + Tm * hF);
        }
    }
}

/* x_eval: the point at which the frozen cells are evaluated (x itself for a record).
 * replay (nullable): a primary hit segment per ray (-1 = none) used instead of the
 * oracle's own closest hit (replay mode: the decision is the given one, the rest FP64). */
static void record2(const o2_scene* s, const o2_params* p, v2 x, v2 x_eval, int64_t rec, const int32_t* replay,
                    double* out) {
    const int N = p->n_dirs;
    const double sig_t = (double)s->sigma_s + (double)s->sigma_a;
    memset(out, 0, sizeof(double) * O2_STRIDE);
    v2* dir = malloc(sizeof(v2) * N);
    double* te = malloc(sizeof(double) * N);
    double* Ls = calloc(3 * (size_t)N, sizeof(double));
    double* dLs = calloc(3 * (size_t)N, sizeof(double));
    double* Lm = calloc(3 * (size_t)N, sizeof(double));
    double* dLm = calloc(3 * (size_t)N, sizeof(double));
    int* cu = calloc((size_t)N, sizeof(int));
    int pnear = 0;
    double tmax = 0.0;
    const double wmc = 2.0 * O2_PI / N, f = 1.0 / (2.0 * O2_PI);
    double bmc[3] = {0, 0, 0};
    for (int j = 0; j < N; ++j) {
        dir[j] = ray_dir2(p, rec, j);
        double t, ne = 1e300;
        int id = -1;
        if (s->circle_mode) {
            t = circle_exit(s, x, dir[j]);
            for (int c = 0; c < 3; ++c) Ls[3 * j + c] = s->circle_Le[c];
            id = 0;
        } else {
            id = closest2(s, x, dir[j], &t, &ne);
            if (replay && replay[j] != id && replay[j] >= -1 && replay[j] < s->n_segs) {
                id = replay[j];
                if (id >= 0) {        /* the given segment's line, its endpoints not tested */
                    v2 e = sub2(seg_b(s, id), seg_a(s, id)), w = sub2(seg_a(s, id), x);
                    double den = crs2(dir[j], e);
                    if (den != 0.0) t = crs2(w, e) / den;
                }
            }
            if (replay) ne = 1e300;
            if (id >= 0) surface_Lo(s, id, add2(x, scl2(dir[j], t)), dir[j], &Ls[3 * j], &dLs[3 * j]);
            else t = square_exit(x, dir[j]);
        }
        if (ne < O2_NEAR) ++pnear;
        te[j] = t;
        if (t > tmax) tmax = t;
        if (id >= 0)
            for (int c = 0; c < 3; ++c) {
                out[O_LSS + c] += wmc * f * exp(-sig_t * t) * Ls[3 * j + c];
                bmc[c] += wmc * f * exp(-sig_t * t) * dLs[3 * j + c];
            }
    }
    int K = (int)ceil(tmax / p->dt);
    out[O_K] = K;
    static const double zero3[3] = {0, 0, 0};
    int ndeg = 0;
    acc2 A[2];
    memset(A, 0, sizeof(A));
    const double wms = (double)s->sigma_s * p->dt;
    for (int k = 0; k <= K; ++k) {
        double tk = ((double)k - 0.5) * p->dt;
        if (k >= 1) {
            for (int j = 0; j < N; ++j) {
                double* lo = &Lm[3 * j];
                double* dlo = &dLm[3 * j];
                lo[0] = lo[1] = lo[2] = dlo[0] = dlo[1] = dlo[2] = 0.0;
                /* a vertex within float rounding of its ray's hit may land on either side */
                cu[j] = fabs(tk - te[j]) < 1e-6 * (1.0 + te[j]);
                if (tk < te[j] || cu[j]) {
                    double Lv[3], dLv[3] = {0, 0, 0};
                    medium_Lo(s, add2(x, scl2(dir[j], tk)), Lv, dLv);
                    for (int c = 0; c < 3; ++c) {
                        if (tk < te[j]) {
                            lo[c] = Lv[c];
                            dlo[c] = dLv[c];
                            out[O_LMS + c] += wmc * f * exp(-sig_t * tk) * lo[c];
                        }
                        if (cu[j]) dlo[c] += fabs(Lv[c]) + dLv[c];
                        bmc[c] += wms * wmc * f * exp(-sig_t * tk) * dlo[c];
                    }
                }
            }
        }
        int part = k == 0 ? 0 : 1;
        double w = k == 0 ? 1.0 : wms;
        for (int j = 0; j < N; ++j) {
            int jj[2] = {j, (j + 1) % N};
            v2 y[2];
            double t[2];
            const double* Lo[2];
            const double* dLo[2];
            int cun[2];
            for (int q = 0; q < 2; ++q) {
                int v = jj[q];
                t[q] = (k == 0 || !(tk < te[v])) ? te[v] : tk;
                y[q] = add2(x, scl2(dir[v], t[q]));
                Lo[q] = k == 0 ? &Ls[3 * v] : ((tk < te[v]) ? &Lm[3 * v] : zero3);
                dLo[q] = k == 0 ? &dLs[3 * v] : &dLm[3 * v];
                cun[q] = k == 0 ? 0 : cu[v];
            }
            cell2(x_eval, y, t, Lo, dLo, cun, sig_t, w, &A[part], &ndeg);
        }
    }
    for (int c = 0; c < 3; ++c) {
        out[O_LMS + c] *= wms;
        out[O_L + c] = out[O_LSS + c] + out[O_LMS + c];
        out[O_LFF + c] = A[0].L[c] + A[1].L[c];
        out[O_BL + c] = bmc[c];
        out[O_BG + c] = A[0].bg[c] + A[1].bg[c];
        out[O_BH + c] = A[0].bh[c] + A[1].bh[c];
    }
    for (int e = 0; e < 6; ++e) {
        out[O_GSS + e] = A[0].g[e];
        out[O_GMS + e] = A[1].g[e];
        out[O_G + e] = A[0].g[e] + A[1].g[e];
    }
    for (int e = 0; e < 9; ++e) {
        out[O_HSS + e] = A[0].h[e];
        out[O_HMS + e] = A[1].h[e];
        out[O_H + e] = A[0].h[e] + A[1].h[e];
    }
    double LY = 0, hY[3] = {0, 0, 0};
    for (int c = 0; c < 3; ++c) {
        LY += LUM2[c] * out[O_L + c];
        for (int e = 0; e < 3; ++e) hY[e] += LUM2[c] * out[O_H + 3 * c + e];
    }
    int status = 0;
    out[O_R] = o2_radius(LY, hY, (double)p->eps, (double)p->r_min, (double)p->r_max, &status, &out[O_EIG]);
    out[O_ST] = status;
    out[O_PNEAR] = pnear;
    free(dir);
    free(te);
    free(Ls);
    free(dLs);
    free(Lm);
    free(dLm);
    free(cu);
}

int o2_stride(void) { return O2_STRIDE; }

/* n records; replay (nullable) gives replay_stride primary hit segment ids per record */
int o2_records(const o2_scene* s, const o2_params* p, const float* pos, const int64_t* rec_ids, int n, double* out,
               const int32_t* replay, int replay_stride) {
    for (int i = 0; i < n; ++i) {
        v2 x = mk2(pos[2 * i], pos[2 * i + 1]);
        int64_t rid = rec_ids ? rec_ids[i] : p->rec_base + i;
        record2(s, p, x, x, rid, replay ? replay + (size_t)i * replay_stride : NULL, out + (size_t)i * O2_STRIDE);
    }
    return 0;
}

/* the record's triangulated radiance with its ray set and shells built at x0 but the
 * cells evaluated at x_eval (for frozen-vertex finite differences) */
int o2_frozen_eval(const o2_scene* s, const o2_params* p, const float* x0, int64_t rec, const double* x_eval,
                   double* out) {
    record2(s, p, mk2(x0[0], x0[1]), mk2(x_eval[0], x_eval[1]), rec, NULL, out);
    return 0;
}

/* primitives for the pins */
int o2_segment_angle(const double* x, const double* y0, const double* y1, double* out6) {
    s2fun F;
    int ok = segment_angle(mk2(x[0], x[1]), mk2(y0[0], y0[1]), mk2(y1[0], y1[1]), &F);
    out6[0] = F.v;
    out6[1] = F.g[0];
    out6[2] = F.g[1];
    out6[3] = F.h[0];
    out6[4] = F.h[1];
    out6[5] = F.h[2];
    return ok;
}

void o2_transmittance(const double* x, const double* y, double sigma_t, double* out6) {
    s2fun T;
    transmittance2(mk2(x[0], x[1]), mk2(y[0], y[1]), sigma_t, &T);
    out6[0] = T.v;
    out6[1] = T.g[0];
    out6[2] = T.g[1];
    out6[3] = T.h[0];
    out6[4] = T.h[1];
    out6[5] = T.h[2];
}

void o2_ray_directions(const o2_params* p, int64_t rec, double* out) {
    for (int j = 0; j < p->n_dirs; ++j) {
        v2 d = ray_dir2(p, rec, j);
        out[2 * j] = d.x;
        out[2 * j + 1] = d.y;
    }
}

void o2_trace(const o2_scene* s, const double* o, const double* d, int n, int32_t* id, double* t) {
    for (int i = 0; i < n; ++i) {
        double tt;
        id[i] = closest2(s, mk2(o[2 * i], o[2 * i + 1]), mk2(d[2 * i], d[2 * i + 1]), &tt, NULL);
        t[i] = tt;
    }
}
