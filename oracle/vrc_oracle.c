/*
 * vrc_oracle.c -- plain FP64 CPU oracle for second-order occlusion-aware
 * volumetric radiance caching (Marco, Jarabo, Jarosz, Gutierrez, TOG 37(2) 2018).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the benchmark's
 * CPU-baseline leg may load this library.  It shares no code, header, table or
 * helper with the CUDA library; the only thing both sides share are the seeded
 * inputs (scenes, positions) and the published splitmix64 generator, which each
 * side implements on its own.
 *
 * Everything is double precision, written for readability: brute-force or a
 * simple median-split BVH for ray casting, per-channel evaluation of the paper's
 * product-rule equations, plain summation, cyclic Jacobi for the eigenvalues.
 *
 * Readings of the paper that this file fixes (where it is silent or garbled):
 *  R1  the cached quantity is L = int f_s L_i dw (Eq. outLF, no sigma_s at x);
 *      sigma_s enters only medium shells through Eq. mediaLFin.
 *  R2  the cell radiance uses the solid angle itself, L_j = f T L_o Omega_j
 *      (Eq. ApproxSegmentRadiance with int G dy = Omega); App. C's F = Omega/4pi
 *      is computed as printed and multiplied by 4pi.
 *  R3  the printed gradient of A in App. C drops a transpose; the correct one is
 *      grad A = -(y2-y1) x (y3-y1), constant in x, so J(grad A) = 0 as App. C states.
 *  R4  "add pi when the arctangent is negative" is Omega = 2 atan2(A, B).
 *  R5  signed A by default (consistent winding closes every shell: sum Omega = 4pi);
 *      ff_signed = 0 gives the printed |A|.
 *  R6  stratification: equal d(cos theta) x equal d(phi) strata, one jittered ray
 *      each, plus two unweighted pole rays; quads split along (i,j)-(i+1,j+1);
 *      every cell wound counter-clockwise seen from outside.
 *  R7  medium shells at t_k = (k - 1/2) dt, k = 1..K, K = ceil(max t_end / dt).
 *  R8  splitmix64 jitter u = (splitmix64(seed ^ rec<<32 ^ i<<16 ^ j ^ stream<<60) >> 40) 2^-24.
 *  R9  the cell's "furthest point" (for T and L_o) is its vertex with the largest ray
 *      parameter t.  When several vertices tie exactly (every unclamped vertex of a
 *      medium shell sits at the same t_k), the cell's reduced radiance L_r = L_o T and
 *      its derivatives are the mean over the tied vertices: any fixed tie-break picks
 *      the same corner of every cell and biases the derivatives to first order in the
 *      cell size.  The vertices are frozen under differentiation.
 *  R10 rays that leave the unit cube without a hit end at the exit with L_o = 0.
 *  R11 vertex radiance: Lambertian two-sided surfaces (light must be on x's side),
 *      single scattering in the medium, both from point lights with shadow rays;
 *      constant per vertex (grad L_o = 0), direction to x taken to the record centre.
 *  R12 direct point-light in-scattering at x itself is not part of the record.
 *  R13 Henyey-Greenstein phase with mu = w_i . w_o, w_i = (x - y_c)/|x - y_c|, y_c the
 *      cell's centroid (Sec. 4 lets w_l point to any point of the cell; the centroid
 *      keeps the phase bias second order), so f depends on x and the general
 *      product-rule equations are used.
 *  R14 the stored radiance is the Monte Carlo estimate (Sec. 4, last paragraph);
 *      the triangulated estimate L_ff is a diagnostic.
 *  R15 isotropic radius from the largest |eigenvalue| of the Rec.709 luminance
 *      Hessian with the MC luminance, clamped to [r_min, r_max].
 *  R16 ray hits: smallest t, then lowest primitive id; t_min = 1e-6; surface
 *      shadow rays start 1e-5 along the normal facing x.
 *  R17 ellipsoidal records: one radius per Hessian eigenvalue (Eq. radiusAniso3D
 *      with |lambda_i|, the same clamps) along its eigenvector; a query's distance
 *      ratio |x' - x_k| / R_k becomes the ellipsoidal norm sqrt(D^T M_k D), with
 *      M_k = sum_i v_i v_i^T / R_i^2, in the membership test and in d = 1 - ratio.
 *  R18 lo_grad (optional, off by default; Sec. 7's extension of R11): an open medium
 *      vertex y scatters its light toward x, so its radiance toward x is
 *      L_o(x_c) f(l . w(x)) / f(l . w(x_c)), l = (y - p_light)/|y - p_light|,
 *      w(x) = (x - y)/|x - y|: the ratio is 1 at the centre and carries grad L_o and
 *      H L_o into the product rule.  One light only (with several, each light's share
 *      of L_o would need its own factor); surface and clamped vertices stay constant.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_PI 3.14159265358979323846
#define ORC_TMIN 1e-6
#define ORC_SHADOW_OFFSET 1e-5
#define ORC_OUT_STRIDE 132

/* output slots of one record (doubles) */
enum {
    O_L = 0, O_L_SS = 3, O_L_MS = 6,
    O_G = 9, O_G_SS = 18, O_G_MS = 27,           /* [channel][axis] */
    O_H = 36, O_H_SS = 54, O_H_MS = 72,          /* [channel][xx,xy,xz,yy,yz,zz] */
    O_LFF = 90, O_R = 93, O_EIG = 94, O_KAPPA = 97, O_STATUS = 98, O_NSHELL = 99,
    O_MEDGE = 100, O_MT = 101, O_NRAYS = 102, O_NDEGEN = 103, O_LFF_SS = 104,
    O_LFF_MS = 107, O_LY = 110, O_LAMMAX = 111,
    /* decision-sensitivity budgets (filled when track_margins = 1): the largest change
     * that flipping every near-tie decision of the record could make */
    O_BUD_L = 112, O_BUD_LFF = 115, O_BUD_G = 118, O_BUD_H = 121, O_N_PRIM_UNC = 124, O_N_UNC = 125,
    /* replay mode: rays whose given primary hit differs from the oracle's own, ids out of range */
    O_N_REPLAYED = 126, O_N_BAD_REPLAY = 127,
    /* full replay: visibility decisions taken the given way (each a near tie here), and
     * given decisions that are not near ties in FP64 (a ray end beyond rounding of the
     * oracle's, a vertex lit or dark with no shadow ray near an edge) */
    O_N_LIT_REPLAYED = 128, O_N_UNEXPLAINED = 129
};

/* The discrete decisions of a record taken from elsewhere (replay mode).  hit: primary hit
 * id per ray (-1 = none); t: the ray's end as computed in FP32, which then decides the
 * clamps of shell vertices (open iff t_k < t, both FP32) and the furthest vertices of each
 * cell (largest such parameter); lit: a bit per (shell, ray), set when the vertex has
 * radiance, which settles each shadow-ray near tie.  t and lit are used together (full
 * replay) or not at all; hit may be given alone. */
typedef struct {
    const int32_t* hit;
    const float* t;
    const uint32_t* lit;
    int stride;        /* rays per record in hit and t */
    int shells;        /* rows of lit per record */
} orc_replay;

/* a discrete decision is "near-tie" when FP32 rounding could flip it */
#ifndef TIE_EDGE
#define TIE_EDGE 1e-6   /* scene units: ray passes this close to a triangle edge */
#endif
#ifndef TIE_T
#define TIE_T 5e-7      /* relative gap between two ray parameters (scaled by 1 + 1/|cos incidence|) */
#endif

/* per-record status bits */
#define REC_NONFINITE 1
#define REC_CLAMP_LO 2
#define REC_CLAMP_HI 4
#define REC_DEGENERATE 8

/* ------------------------------------------------------------------ inputs */
typedef struct {
    int n_tris;
    const float* tri_v;      /* [n_tris][3][3] */
    const float* albedo;     /* [n_tris][3] */
    const float* emission;   /* [n_tris][3] or NULL */
    float sigma_s, sigma_a, g;
    int n_lights;
    const float* light_pos;  /* [n_lights][3] */
    const float* light_I;    /* [n_lights][3] */
    int use_bvh;             /* 0: brute force over all triangles */
    int sphere_mode;         /* test mode: analytic sphere around the record, constant radiance */
    float sphere_c[3];
    float sphere_r;
    float sphere_Le[3];
} orc_scene_in;

typedef struct {
    int n_bands, n_bins;
    float dt, eps;
    float omega_o[3];
    uint64_t seed;
    int ff_signed;
    int extrap_order;
    float r_min, r_max;
    int64_t rec_base;
    int general_derivs;      /* 1: Eqs. SSSegALGradient/Hessian; 0: simplified Eqs. (g = 0) */
    int track_margins;       /* 1: record decision margins (slower) */
    int surface_only;        /* 1: skip medium shells (closed-form sphere test) */
    int lo_grad;             /* 1: keep grad L_o of medium vertices (one light; see cell_radiance) */
} orc_params;

/* ------------------------------------------------------------ vector utils */
typedef struct { double x, y, z; } v3;
static inline v3 mk(double x, double y, double z) { v3 r = {x, y, z}; return r; }
static inline v3 add(v3 a, v3 b) { return mk(a.x + b.x, a.y + b.y, a.z + b.z); }
static inline v3 sub(v3 a, v3 b) { return mk(a.x - b.x, a.y - b.y, a.z - b.z); }
static inline v3 scl(v3 a, double s) { return mk(a.x * s, a.y * s, a.z * s); }
static inline double dot(v3 a, v3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
static inline v3 cross(v3 a, v3 b) {
    return mk(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}
static inline double norm(v3 a) { return sqrt(dot(a, a)); }
static inline double comp(v3 a, int i) { return i == 0 ? a.x : (i == 1 ? a.y : a.z); }
static inline v3 ldv(const float* p) { return mk((double)p[0], (double)p[1], (double)p[2]); }

/* scalar function of x with its gradient and full 3x3 Hessian */
typedef struct { double v; double g[3]; double H[3][3]; } sfun;

static void outer_add(double H[3][3], double s, v3 a, v3 b) {
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) H[i][j] += s * comp(a, i) * comp(b, j);
}
static void ident_add(double H[3][3], double s) { for (int i = 0; i < 3; ++i) H[i][i] += s; }

/* ---------------------------------------------- jitter (reading R8) */
static uint64_t splitmix64(uint64_t x) {
    /* Steele, Lea, Flood (OOPSLA 2014) finaliser as published by Vigna. */
    uint64_t z = x + 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}
static double jitter(uint64_t seed, int64_t rec, int i, int j, int stream) {
    uint64_t key = seed ^ ((uint64_t)rec << 32) ^ ((uint64_t)i << 16) ^ (uint64_t)j ^
                   ((uint64_t)stream << 60);
    return (double)(splitmix64(key) >> 40) * (1.0 / 16777216.0);
}

/* ---------------------------------------------- ray set (Sec. 6 Implementation, R6) */
static v3 ray_direction(const orc_params* p, int nb, int ns, int64_t rec, int v) {
    int n = nb * ns;
    if (v == n) return mk(0, 0, 1);
    if (v == n + 1) return mk(0, 0, -1);
    int i = v / ns, j = v % ns;
    double u1 = jitter(p->seed, rec, i, j, 0), u2 = jitter(p->seed, rec, i, j, 1);
    double ct = 1.0 - 2.0 * ((double)i + u1) / (double)nb;
    double st = sqrt(fmax(0.0, 1.0 - ct * ct));
    double ph = 2.0 * ORC_PI * ((double)j + u2) / (double)ns;
    return mk(st * cos(ph), st * sin(ph), ct);
}

/* ------------------------------------------------------------- scene + BVH */
typedef struct { v3 a, b, c; int id; int seamless[3]; /* edge ab, bc, ca joins a coplanar twin */ } otri;
typedef struct { double lo[3], hi[3]; int left, right, start, count; } onode;

typedef struct {
    orc_scene_in in;
    int n;
    otri* tri;        /* in BVH leaf order */
    onode* node;
    int n_nodes;
    double sigma_t;
} orc_scene;

#define BVH_PAD 2e-4   /* boxes padded so near misses within the margin radius are visited */

static int cmp_axis;
static const otri* cmp_tris;
static double centroid(const otri* t, int ax) { return (comp(t->a, ax) + comp(t->b, ax) + comp(t->c, ax)) / 3.0; }
static int cmp_tri(const void* a, const void* b) {
    double ca = centroid((const otri*)a, cmp_axis), cb = centroid((const otri*)b, cmp_axis);
    if (ca < cb) return -1;
    if (ca > cb) return 1;
    return ((const otri*)a)->id - ((const otri*)b)->id;
}

static int bvh_build(orc_scene* s, int start, int count) {
    int me = s->n_nodes++;
    onode* nd = &s->node[me];
    for (int k = 0; k < 3; ++k) { nd->lo[k] = 1e300; nd->hi[k] = -1e300; }
    double clo[3] = {1e300, 1e300, 1e300}, chi[3] = {-1e300, -1e300, -1e300};
    for (int t = start; t < start + count; ++t) {
        const otri* T = &s->tri[t];
        v3 p[3] = {T->a, T->b, T->c};
        for (int q = 0; q < 3; ++q)
            for (int k = 0; k < 3; ++k) {
                nd->lo[k] = fmin(nd->lo[k], comp(p[q], k) - BVH_PAD);
                nd->hi[k] = fmax(nd->hi[k], comp(p[q], k) + BVH_PAD);
            }
        for (int k = 0; k < 3; ++k) {
            double c = centroid(T, k);
            clo[k] = fmin(clo[k], c);
            chi[k] = fmax(chi[k], c);
        }
    }
    if (count <= 4) {
        nd->left = nd->right = -1;
        nd->start = start;
        nd->count = count;
        return me;
    }
    int ax = 0;
    for (int k = 1; k < 3; ++k)
        if (chi[k] - clo[k] > chi[ax] - clo[ax]) ax = k;
    cmp_axis = ax;  /* single-threaded build */
    cmp_tris = s->tri;
    qsort(&s->tri[start], (size_t)count, sizeof(otri), cmp_tri);
    int half = count / 2;
    nd->start = start;
    nd->count = 0;
    int l = bvh_build(s, start, half);
    int r = bvh_build(s, start + half, count - half);
    s->node[me].left = l;
    s->node[me].right = r;
    return me;
}

static void mark_seamless(orc_scene* s);
static int same_surface(const orc_scene* s, int i, int j);

orc_scene* orc_scene_create(const orc_scene_in* in) {
    orc_scene* s = (orc_scene*)calloc(1, sizeof(orc_scene));
    s->in = *in;
    s->n = in->n_tris;
    s->sigma_t = (double)in->sigma_s + (double)in->sigma_a;
    s->tri = (otri*)calloc((size_t)(s->n > 0 ? s->n : 1), sizeof(otri));
    for (int t = 0; t < s->n; ++t) {
        s->tri[t].a = ldv(in->tri_v + 9 * t);
        s->tri[t].b = ldv(in->tri_v + 9 * t + 3);
        s->tri[t].c = ldv(in->tri_v + 9 * t + 6);
        s->tri[t].id = t;
    }
    if (s->n > 0) mark_seamless(s);
    s->node = (onode*)calloc((size_t)(2 * (s->n > 0 ? s->n : 1) + 1), sizeof(onode));
    s->n_nodes = 0;
    if (in->use_bvh && s->n > 0) bvh_build(s, 0, s->n);
    return s;
}

/* two triangles render identically where they meet: coplanar, same material */
static int same_surface(const orc_scene* s, int i, int j) {
    const orc_scene_in* in = &s->in;
    v3 a = ldv(in->tri_v + 9 * i), b = ldv(in->tri_v + 9 * i + 3), c = ldv(in->tri_v + 9 * i + 6);
    v3 p = ldv(in->tri_v + 9 * j), q = ldv(in->tri_v + 9 * j + 3), r = ldv(in->tri_v + 9 * j + 6);
    v3 n1 = cross(sub(b, a), sub(c, a)), n2 = cross(sub(q, p), sub(r, p));
    if (norm(cross(n1, n2)) > 1e-9 * norm(n1) * norm(n2)) return 0;
    if (fabs(dot(n1, sub(p, a))) > 1e-9 * norm(n1)) return 0;
    for (int k = 0; k < 3; ++k) {
        if (in->albedo[3 * i + k] != in->albedo[3 * j + k]) return 0;
        if (in->emission && in->emission[3 * i + k] != in->emission[3 * j + k]) return 0;
    }
    return 1;
}

typedef struct { double k[6]; int tri, e; } edgekey;
static int cmp_edge(const void* x, const void* y) {
    const edgekey *a = (const edgekey*)x, *b = (const edgekey*)y;
    for (int i = 0; i < 6; ++i) {
        if (a->k[i] < b->k[i]) return -1;
        if (a->k[i] > b->k[i]) return 1;
    }
    return 0;
}
static int cmp_v3(v3 a, v3 b) {
    if (a.x != b.x) return a.x < b.x ? -1 : 1;
    if (a.y != b.y) return a.y < b.y ? -1 : 1;
    if (a.z != b.z) return a.z < b.z ? -1 : 1;
    return 0;
}

/* mark every edge shared (same endpoints) with a coplanar triangle of the same material */
static void mark_seamless(orc_scene* s) {
    int n = s->n;
    edgekey* E = (edgekey*)malloc(sizeof(edgekey) * (size_t)(3 * n + 1));
    for (int t = 0; t < n; ++t) {
        const otri* T = &s->tri[t];
        v3 p[3] = {T->a, T->b, T->c};
        for (int e = 0; e < 3; ++e) {
            v3 u = p[e], w = p[(e + 1) % 3];
            if (cmp_v3(u, w) > 0) { v3 tmp = u; u = w; w = tmp; }
            edgekey* K = &E[3 * t + e];
            K->k[0] = u.x; K->k[1] = u.y; K->k[2] = u.z; K->k[3] = w.x; K->k[4] = w.y; K->k[5] = w.z;
            K->tri = t;
            K->e = e;
        }
    }
    qsort(E, (size_t)(3 * n), sizeof(edgekey), cmp_edge);
    for (int i = 0; i < 3 * n;) {
        int j = i + 1;
        while (j < 3 * n && cmp_edge(&E[i], &E[j]) == 0) ++j;
        for (int a = i; a < j; ++a)
            for (int b = i; b < j; ++b)
                if (a != b && same_surface(s, s->tri[E[a].tri].id, s->tri[E[b].tri].id))
                    s->tri[E[a].tri].seamless[E[a].e] = 1;
        i = j;
    }
    free(E);
}

void orc_scene_destroy(orc_scene* s) {
    if (!s) return;
    free(s->tri);
    free(s->node);
    free(s);
}

/* --------------------------------------------------------- ray casting (R16) */
typedef struct {
    double t;         /* best t so far */
    int id;           /* best primitive id, -1 none */
    double margin;    /* min distance of a near-boundary crossing to a triangle edge */
    double tie;       /* min relative t gap between the hit and another hit */
    double limit;     /* segment end for any-hit / margin queries */
    double tie_val;   /* as tie, counting only hits on a different surface (value-affecting) */
    const orc_scene* s;
} hitrec;

static double seg_dist(v3 p, v3 a, v3 b) {
    v3 ab = sub(b, a);
    double L2 = dot(ab, ab);
    double s = L2 > 0 ? dot(sub(p, a), ab) / L2 : 0.0;
    s = s < 0 ? 0 : (s > 1 ? 1 : s);
    return norm(sub(p, add(a, scl(ab, s))));
}

/* Moller-Trumbore in double: plane parameter t and barycentrics (u, v). */
static int mt(v3 o, v3 d, const otri* T, double* t, double* u, double* v) {
    v3 e1 = sub(T->b, T->a), e2 = sub(T->c, T->a);
    v3 p = cross(d, e2);
    double det = dot(e1, p);
    if (fabs(det) < 1e-300) return 0;
    double inv = 1.0 / det;
    v3 s = sub(o, T->a);
    *u = dot(s, p) * inv;
    v3 q = cross(s, e1);
    *v = dot(d, q) * inv;
    *t = dot(e2, q) * inv;
    return 1;
}

static void test_tri_closest(v3 o, v3 d, const otri* T, hitrec* h) {
    double t, u, v;
    if (!mt(o, d, T, &t, &u, &v)) return;
    if (u >= 0 && v >= 0 && u + v <= 1 && t > ORC_TMIN) {
        if (t < h->t || (t == h->t && T->id < h->id)) { h->t = t; h->id = T->id; }
    }
}

static void test_tri_any(v3 o, v3 d, const otri* T, hitrec* h) {
    double t, u, v;
    if (!mt(o, d, T, &t, &u, &v)) return;
    if (u >= 0 && v >= 0 && u + v <= 1 && t > ORC_TMIN && t < h->limit) h->id = T->id;
}

/* margin bookkeeping: crossings of the segment (tmin, limit] that pass within
 * 1e-4 of a triangle's boundary (edges joining a coplanar twin of the same material
 * are seamless and do not count), and near-equal t between distinct hits */
static void test_tri_margin(v3 o, v3 d, const otri* T, hitrec* h, int best_id, double best_t) {
    double t, u, v;
    if (!mt(o, d, T, &t, &u, &v)) return;
    if (!(t > ORC_TMIN * 0.5 && t <= h->limit * (1.0 + 1e-6) + 1e-9)) return;
    double w = 1.0 - u - v;
    if (u < -0.05 || v < -0.05 || w < -0.05) return;
    v3 p = add(o, scl(d, t));
    double e = INFINITY;
    if (!T->seamless[0]) e = fmin(e, seg_dist(p, T->a, T->b));
    if (!T->seamless[1]) e = fmin(e, seg_dist(p, T->b, T->c));
    if (!T->seamless[2]) e = fmin(e, seg_dist(p, T->c, T->a));
    if (e < 1e-4 && e < h->margin) h->margin = e;      /* only near misses count (boxes are padded 2e-4) */
    if (best_id >= 0 && T->id != best_id && u >= 0 && v >= 0 && w >= 0) {
        double gap = fabs(t - best_t) / fmax(best_t, 1e-30);
        if (gap < h->tie) h->tie = gap;
        if (gap < h->tie_val && !same_surface(h->s, T->id, best_id)) h->tie_val = gap;
    }
}

static int box_hit(const onode* n, v3 o, v3 inv, double tmax) {
    double t0 = 0.0, t1 = tmax;
    for (int k = 0; k < 3; ++k) {
        double ok = comp(o, k), ik = comp(inv, k);
        double a = (n->lo[k] - ok) * ik, b = (n->hi[k] - ok) * ik;
        if (isnan(a)) a = -INFINITY;
        if (isnan(b)) b = INFINITY;
        if (a > b) { double tt = a; a = b; b = tt; }
        if (a > t0) t0 = a;
        if (b < t1) t1 = b;
        if (t0 > t1) return 0;
    }
    return 1;
}

enum { Q_CLOSEST, Q_ANY, Q_MARGIN };

static void traverse(const orc_scene* s, v3 o, v3 d, hitrec* h, int mode, int best_id, double best_t) {
    if (s->n == 0) return;
    if (!s->in.use_bvh) {
        for (int t = 0; t < s->n; ++t) {
            if (mode == Q_CLOSEST) test_tri_closest(o, d, &s->tri[t], h);
            else if (mode == Q_ANY) { test_tri_any(o, d, &s->tri[t], h); if (h->id >= 0) return; }
            else test_tri_margin(o, d, &s->tri[t], h, best_id, best_t);
        }
        return;
    }
    v3 inv = mk(1.0 / d.x, 1.0 / d.y, 1.0 / d.z);
    int stack[128];
    int sp = 0;
    stack[sp++] = 0;
    while (sp) {
        const onode* n = &s->node[stack[--sp]];
        double tmax = mode == Q_CLOSEST ? h->t : h->limit * (1.0 + 1e-6) + 1e-9;
        if (!box_hit(n, o, inv, tmax)) continue;
        if (n->left < 0) {
            for (int t = n->start; t < n->start + n->count; ++t) {
                if (mode == Q_CLOSEST) test_tri_closest(o, d, &s->tri[t], h);
                else if (mode == Q_ANY) { test_tri_any(o, d, &s->tri[t], h); if (h->id >= 0) return; }
                else test_tri_margin(o, d, &s->tri[t], h, best_id, best_t);
            }
        } else {
            stack[sp++] = n->left;
            stack[sp++] = n->right;
        }
    }
}

/* closest hit with t > t_min (unbounded); returns id or -1 */
static int closest_hit(const orc_scene* s, v3 o, v3 d, double* t_out, double* margin, double* tie, double* tie_val,
                       int track) {
    hitrec h = {INFINITY, -1, INFINITY, INFINITY, INFINITY, INFINITY, s};
    traverse(s, o, d, &h, Q_CLOSEST, -1, 0);
    if (track) {
        hitrec m = {0, -1, INFINITY, INFINITY, h.id >= 0 ? h.t : 4.0, INFINITY, s};
        traverse(s, o, d, &m, Q_MARGIN, h.id, h.t);
        *margin = m.margin;
        *tie = m.tie;
        *tie_val = m.tie_val;
    }
    *t_out = h.t;
    return h.id;
}

/* 1 if any triangle crosses the open segment (t_min, limit) */
static int occluded(const orc_scene* s, v3 o, v3 d, double limit, double* margin, int track) {
    hitrec h = {0, -1, INFINITY, INFINITY, limit, INFINITY, s};
    traverse(s, o, d, &h, Q_ANY, -1, 0);
    if (track) {
        hitrec m = {0, -1, INFINITY, INFINITY, limit, INFINITY, s};
        traverse(s, o, d, &m, Q_MARGIN, -1, 0);
        if (m.margin < *margin) *margin = m.margin;
    }
    return h.id >= 0;
}

/* distance to leave the unit cube (R10) */
static double cube_exit(v3 x, v3 d) {
    double t = INFINITY;
    for (int k = 0; k < 3; ++k) {
        double xk = comp(x, k), dk = comp(d, k);
        if (dk > 0) t = fmin(t, (1.0 - xk) / dk);
        else if (dk < 0) t = fmin(t, -xk / dk);
    }
    return t;
}

/* ------------------------------------------- phase function (Henyey-Greenstein) */
double orc_hg(double mu, double g) {
    return (1.0 - g * g) / (4.0 * ORC_PI * pow(1.0 + g * g - 2.0 * g * mu, 1.5));
}

/* ---------------------------------------------------- vertex radiance (R11) */
/* Vertex radiance with its shadow-ray decisions.  When track is set, every light whose
 * shadow ray passes within TIE_EDGE of a triangle edge (a decision FP32 may take the
 * other way) adds |its term| to dLo, its signed change if the ray went the other way
 * to sLo, and 1 to *nsh.  dLo, sLo and nsh may be NULL when track is 0. */
static void surface_radiance(const orc_scene* s, int id, v3 y, v3 d, double Lo[3], double dLo[3], double sLo[3],
                             int* nsh, int track) {
    const orc_scene_in* in = &s->in;
    Lo[0] = Lo[1] = Lo[2] = 0.0;
    if (in->emission)
        for (int c = 0; c < 3; ++c) Lo[c] += (double)in->emission[3 * id + c];
    v3 a = ldv(in->tri_v + 9 * id), b = ldv(in->tri_v + 9 * id + 3), cc = ldv(in->tri_v + 9 * id + 6);
    v3 n = cross(sub(b, a), sub(cc, a));
    n = scl(n, 1.0 / norm(n));
    if (dot(n, d) > 0) n = scl(n, -1.0);        /* two-sided: face the record centre */
    for (int L = 0; L < in->n_lights; ++L) {
        v3 pl = ldv(in->light_pos + 3 * L);
        v3 l = sub(pl, y);
        double dist = norm(l);
        v3 lh = scl(l, 1.0 / dist);
        double cs = dot(n, lh);
        if (cs <= 0) continue;                    /* light on the far side */
        v3 o = add(y, scl(n, ORC_SHADOW_OFFSET));
        v3 lo = sub(pl, o);
        double dl = norm(lo);
        double margin = INFINITY;
        int occ = occluded(s, o, scl(lo, 1.0 / dl), dl, &margin, track);
        double T = exp(-s->sigma_t * dist);
        int near = track && margin < TIE_EDGE;
        for (int c = 0; c < 3; ++c) {
            double v = (double)in->albedo[3 * id + c] / ORC_PI * (double)in->light_I[3 * L + c] * cs * T / (dist * dist);
            if (!occ) Lo[c] += v;
            if (near) { dLo[c] += fabs(v); sLo[c] += occ ? v : -v; }
        }
        if (near) ++*nsh;
    }
}

static void medium_radiance(const orc_scene* s, v3 y, v3 d, double Lo[3], double dLo[3], double sLo[3], int* nsh,
                            int track) {
    const orc_scene_in* in = &s->in;
    Lo[0] = Lo[1] = Lo[2] = 0.0;
    for (int L = 0; L < in->n_lights; ++L) {
        v3 pl = ldv(in->light_pos + 3 * L);
        v3 l = sub(pl, y);
        double dist = norm(l);
        v3 lh = scl(l, 1.0 / dist);
        double margin = INFINITY;
        int occ = occluded(s, y, lh, dist, &margin, track);
        /* light travels p_L -> y (direction -lh), scatters toward x (direction -d) */
        double mu = dot(lh, d);
        double f = orc_hg(mu, (double)in->g);
        double T = exp(-s->sigma_t * dist);
        int near = track && margin < TIE_EDGE;
        for (int c = 0; c < 3; ++c) {
            double v = f * (double)in->light_I[3 * L + c] * T / (dist * dist);
            if (!occ) Lo[c] += v;
            if (near) { dLo[c] += fabs(v); sLo[c] += occ ? v : -v; }
        }
        if (near) ++*nsh;
    }
}

/* ------------------------------------- App. A: homogeneous transmittance */
static void transmittance(v3 x, v3 y, double sigma_t, sfun* T) {
    v3 yx = sub(x, y);
    double r = norm(yx);
    memset(T, 0, sizeof(*T));
    T->v = exp(-sigma_t * r);
    for (int i = 0; i < 3; ++i) T->g[i] = -sigma_t * comp(yx, i) / r * T->v;
    /* H T = -sigma_t ( J(yx)/r - yx yx^T / r^3 - sigma_t yx yx^T / r^2 ) T,  J(yx) = I */
    ident_add(T->H, 1.0 / r);
    outer_add(T->H, -1.0 / (r * r * r), yx, yx);
    outer_add(T->H, -sigma_t / (r * r), yx, yx);
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) T->H[i][j] *= -sigma_t * T->v;
}

/* --------------------- phase function as a function of x (general eqs., R13) */
static void phase(v3 x, v3 yl, v3 wo, double g, sfun* f) {
    v3 w = sub(x, yl);
    double r = norm(w);
    v3 wi = scl(w, 1.0 / r);
    double mu = dot(wi, wo);
    double q = 1.0 + g * g - 2.0 * g * mu;
    double c = (1.0 - g * g) / (4.0 * ORC_PI);
    double f0 = c * pow(q, -1.5);
    double f1 = 3.0 * g * c * pow(q, -2.5);       /* df/dmu */
    double f2 = 15.0 * g * g * c * pow(q, -3.5);  /* d2f/dmu2 */
    v3 gmu = scl(sub(wo, scl(wi, mu)), 1.0 / r);  /* grad mu = (w_o - mu w_i) / r */
    double Hmu[3][3] = {{0}};                     /* (-w_o w_i^T - w_i w_o^T - mu I + 3 mu w_i w_i^T) / r^2 */
    outer_add(Hmu, -1.0 / (r * r), wo, wi);
    outer_add(Hmu, -1.0 / (r * r), wi, wo);
    ident_add(Hmu, -mu / (r * r));
    outer_add(Hmu, 3.0 * mu / (r * r), wi, wi);
    memset(f, 0, sizeof(*f));
    f->v = f0;
    for (int i = 0; i < 3; ++i) f->g[i] = f1 * comp(gmu, i);
    outer_add(f->H, f2, gmu, gmu);
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) f->H[i][j] += f1 * Hmu[i][j];
}

/* --------------- App. C: triangle form factor F = Omega / 4pi and derivatives */
static int formfactor(v3 x, v3 y1, v3 y2, v3 y3, int ff_signed, sfun* F) {
    v3 r[3] = {sub(y1, x), sub(y2, x), sub(y3, x)};
    double rho[3] = {norm(r[0]), norm(r[1]), norm(r[2])};
    double A = dot(r[0], cross(r[1], r[2]));
    double B = rho[0] * rho[1] * rho[2] + dot(r[0], r[1]) * rho[2] + dot(r[1], r[2]) * rho[0] +
               dot(r[0], r[2]) * rho[1];
    v3 gA = scl(cross(sub(y2, y1), sub(y3, y1)), -1.0);   /* reading R3; J(grad A) = 0 */
    if (!ff_signed) {
        if (A < 0) { A = -A; gA = scl(gA, -1.0); }        /* grad|A| = sign(A) grad A */
    }
    /* grad rho = -r / rho ;  J(grad rho) = I / rho - r r^T / rho^3 */
    v3 grho[3];
    double Jrho[3][3][3];
    for (int i = 0; i < 3; ++i) {
        grho[i] = scl(r[i], -1.0 / rho[i]);
        memset(Jrho[i], 0, sizeof(Jrho[i]));
        ident_add(Jrho[i], 1.0 / rho[i]);
        outer_add(Jrho[i], -1.0 / (rho[i] * rho[i] * rho[i]), r[i], r[i]);
    }
    /* grad B = grad(rho1 rho2 rho3) + sum over (i,j,k) of grad((r_i . r_j) rho_k) */
    double gB[3] = {0, 0, 0};
    double JB[3][3] = {{0}};
    for (int a = 0; a < 3; ++a) {
        int b = (a + 1) % 3, c = (a + 2) % 3;
        for (int q = 0; q < 3; ++q) gB[q] += rho[b] * rho[c] * comp(grho[a], q);
        /* J grad(rho1 rho2 rho3): rho_b rho_c J(grad rho_a) + rho_a (grad rho_b grad rho_c^T + grad rho_c grad rho_b^T) */
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) JB[i][j] += rho[b] * rho[c] * Jrho[a][i][j];
        outer_add(JB, rho[a], grho[b], grho[c]);
        outer_add(JB, rho[a], grho[c], grho[b]);
    }
    const int pairs[3][3] = {{0, 1, 2}, {1, 2, 0}, {0, 2, 1}};   /* (i, j, k) */
    for (int p = 0; p < 3; ++p) {
        int i = pairs[p][0], j = pairs[p][1], k = pairs[p][2];
        double rij = dot(r[i], r[j]);
        v3 s = add(r[i], r[j]);
        /* grad((r_i.r_j) rho_k) = (r_i.r_j) grad rho_k - rho_k (r_i + r_j) */
        for (int q = 0; q < 3; ++q) gB[q] += rij * comp(grho[k], q) - rho[k] * comp(s, q);
        /* J = (r_i.r_j) J(grad rho_k) + 2 rho_k I - grad rho_k (r_i+r_j)^T - (r_i+r_j) grad rho_k^T */
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) JB[a][b] += rij * Jrho[k][a][b];
        ident_add(JB, 2.0 * rho[k]);
        outer_add(JB, -1.0, grho[k], s);
        outer_add(JB, -1.0, s, grho[k]);
    }
    double D = A * A + B * B;
    memset(F, 0, sizeof(*F));
    if (!(D > 1e-300)) return 0;
    F->v = 2.0 * atan2(A, B) / (4.0 * ORC_PI);            /* reading R4 */
    v3 gBv = mk(gB[0], gB[1], gB[2]);
    v3 N = sub(scl(gA, B), scl(gBv, A));                  /* B grad A - A grad B */
    for (int q = 0; q < 3; ++q) F->g[q] = comp(N, q) / (2.0 * ORC_PI * D);
    /* H F = 1/2pi [ (grad A grad B^T - grad B grad A^T)/D + (B J(grad A) - A J(grad B))/D
     *              - (B grad A - A grad B)(grad A^2 + grad B^2)^T / D^2 ],  J(grad A) = 0 */
    v3 gD = add(scl(gA, 2.0 * A), scl(gBv, 2.0 * B));
    double H[3][3] = {{0}};
    outer_add(H, 1.0 / D, gA, gBv);
    outer_add(H, -1.0 / D, gBv, gA);
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) H[i][j] += -A * JB[i][j] / D;
    outer_add(H, -1.0 / (D * D), N, gD);
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) F->H[i][j] = H[i][j] / (2.0 * ORC_PI);
    return 1;
}

/* ------------------------------------------- one cell's radiance and derivatives
 * Eq. ApproxSegmentRadiance: L_j = f L_r Omega_j (R2) with the reduced radiance
 * L_r = L_o T taken at the furthest vertex (mean over exactly tied furthest vertices,
 * R9) and f along the direction to the cell centroid (R13).  Derivatives by Eqs.
 * SSSegALGradient .. reducedRadianceDerivatives (general; grad L_o = H L_o = 0) or by
 * the simplified Eqs. SSSegALGradientSimp/HessianSimp (isotropic: grad f = H f = 0). */
typedef struct { double L[3]; double g[3][3]; double H[3][3][3]; } cellout;

/* Outgoing radiance of a furthest vertex as a function of x (the extension beyond Sec. 4's
 * grad L_o = 0 that Sec. 7 discusses): a medium vertex scatters its light with the HG phase,
 * so its radiance toward x is L_o(x) = L_o(x_c) f(l . w(x)) / f(l . w(x_c)), l the light's
 * propagation direction at the vertex, w(x) the unit direction from the vertex to x, x_c the
 * record centre where L_o was computed.  lp_far[q] = l and f0_far[q] = f(l . w(x_c)) per
 * furthest vertex (f0 <= 0: constant L_o, as for Lambertian surfaces); NULL: all constant. */
static int cell_radiance(v3 x, v3 y1, v3 y2, v3 y3, int n_far, const v3* y_far, const double* const* Lo_far,
                         double sigma_t, double g, v3 wo, double weight, int general, int ff_signed, cellout* out,
                         const v3* lp_far, const double* f0_far) {
    sfun F, f;
    memset(out, 0, sizeof(*out));
    int ok = formfactor(x, y1, y2, y3, ff_signed, &F);
    /* reading R2: the cell integral of the geometry term is Omega = 4 pi F */
    F.v *= 4.0 * ORC_PI;
    for (int i = 0; i < 3; ++i) {
        F.g[i] *= 4.0 * ORC_PI;
        for (int j = 0; j < 3; ++j) F.H[i][j] *= 4.0 * ORC_PI;
    }
    v3 yc = scl(add(add(y1, y2), y3), 1.0 / 3.0);
    phase(x, yc, wo, g, &f);
    for (int c = 0; c < 3; ++c) {
        /* reduced radiance L_r = L_o T (Eq. reducedRadianceDerivatives with grad L_o = 0),
         * averaged over the tied furthest vertices */
        double Lr = 0.0, gLr[3] = {0, 0, 0}, HLr[3][3] = {{0}};
        for (int q = 0; q < n_far; ++q) {
            sfun T;
            transmittance(x, y_far[q], sigma_t, &T);
            if (lp_far && f0_far && f0_far[q] > 0.0) {
                /* Eq. reducedRadianceDerivatives with grad L_o kept: T u, u = L_o(x) / L_o(x_c) */
                sfun fv, Tu;
                phase(x, y_far[q], lp_far[q], g, &fv);
                double iu = 1.0 / f0_far[q];
                Tu.v = T.v * fv.v * iu;
                for (int i = 0; i < 3; ++i) Tu.g[i] = (T.v * fv.g[i] + fv.v * T.g[i]) * iu;
                for (int i = 0; i < 3; ++i)
                    for (int j = 0; j < 3; ++j)
                        Tu.H[i][j] = (T.v * fv.H[i][j] + T.g[i] * fv.g[j] + fv.g[i] * T.g[j] + fv.v * T.H[i][j]) * iu;
                T = Tu;
            }
            double lo = Lo_far[q][c] * weight / (double)n_far;
            Lr += lo * T.v;
            for (int i = 0; i < 3; ++i) gLr[i] += lo * T.g[i];
            for (int i = 0; i < 3; ++i)
                for (int j = 0; j < 3; ++j) HLr[i][j] += lo * T.H[i][j];
        }
        /* scaled radiance L_F = F L_r (Eq. scaledRadianceDerivatives) */
        double LF = F.v * Lr, gLF[3], HLF[3][3];
        for (int i = 0; i < 3; ++i) gLF[i] = Lr * F.g[i] + gLr[i] * F.v;
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j)
                HLF[i][j] = Lr * F.H[i][j] + gLr[i] * F.g[j] + F.g[i] * gLr[j] + HLr[i][j] * F.v;
        out->L[c] = LF * f.v;
        if (general) {
            /* L_j = L_F f (Eqs. SSSegALGradient, SSSegALHessian) */
            for (int i = 0; i < 3; ++i) out->g[c][i] = LF * f.g[i] + gLF[i] * f.v;
            for (int i = 0; i < 3; ++i)
                for (int j = 0; j < 3; ++j)
                    out->H[c][i][j] = LF * f.H[i][j] + gLF[i] * f.g[j] + f.g[i] * gLF[j] + HLF[i][j] * f.v;
        } else {
            /* isotropic simplification (Eqs. SSSegALGradientSimp, SSSegALHessianSimp) */
            for (int i = 0; i < 3; ++i) out->g[c][i] = f.v * gLF[i];
            for (int i = 0; i < 3; ++i)
                for (int j = 0; j < 3; ++j) out->H[c][i][j] = f.v * HLF[i][j];
        }
    }
    return ok;
}

/* ------------------------------------------------ cell topology (R6) */
/* returns the three vertex indices of cell c of a band x bin triangulation */
static void cell_vertices(int nb, int ns, int c, int* a, int* b, int* d) {
    int n = nb * ns;
    if (c < ns) {                                    /* north cap fan */
        *a = n; *b = c; *d = (c + 1) % ns;
        return;
    }
    c -= ns;
    int nq = 2 * ns * (nb - 1);
    if (c < nq) {
        int q = c / 2, i = q / ns, j = q % ns, j1 = (j + 1) % ns;
        int v00 = i * ns + j, v01 = i * ns + j1, v10 = (i + 1) * ns + j, v11 = (i + 1) * ns + j1;
        if ((c & 1) == 0) { *a = v00; *b = v10; *d = v11; }
        else { *a = v00; *b = v11; *d = v01; }
        return;
    }
    c -= nq;                                         /* south cap fan */
    *a = n + 1;
    *b = (nb - 1) * ns + (c + 1) % ns;
    *d = (nb - 1) * ns + c;
}

int orc_cell_vertices(int nb, int ns, int c, int* out3) {
    cell_vertices(nb, ns, c, &out3[0], &out3[1], &out3[2]);
    return 2 * nb * ns;
}

/* ------------------------------------------------ eigenvalues and radius */
/* cyclic Jacobi rotations; lam ascending, V (if not NULL) gets the matching unit
 * eigenvectors as its columns: H V[:, i] = lam[i] V[:, i] */
static void jacobi3v(const double Hin[3][3], double lam[3], double V[3][3]) {
    double a[3][3], U[3][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
    memcpy(a, Hin, sizeof(a));
    for (int sweep = 0; sweep < 100; ++sweep) {
        double off = fabs(a[0][1]) + fabs(a[0][2]) + fabs(a[1][2]);
        double scale = fabs(a[0][0]) + fabs(a[1][1]) + fabs(a[2][2]) + off;
        if (off <= 1e-15 * scale || off == 0.0) break;
        for (int p = 0; p < 2; ++p)
            for (int q = p + 1; q < 3; ++q) {
                if (a[p][q] == 0.0) continue;
                double th = 0.5 * atan2(2.0 * a[p][q], a[q][q] - a[p][p]);
                double c = cos(th), s = sin(th);
                double b[3][3];
                memcpy(b, a, sizeof(b));
                for (int k = 0; k < 3; ++k) {          /* a <- R^T a R for rotation in (p, q) */
                    b[k][p] = c * a[k][p] - s * a[k][q];
                    b[k][q] = s * a[k][p] + c * a[k][q];
                }
                double e[3][3];
                memcpy(e, b, sizeof(e));
                for (int k = 0; k < 3; ++k) {
                    e[p][k] = c * b[p][k] - s * b[q][k];
                    e[q][k] = s * b[p][k] + c * b[q][k];
                }
                memcpy(a, e, sizeof(a));
                for (int k = 0; k < 3; ++k) {          /* U <- U R */
                    double up = U[k][p], uq = U[k][q];
                    U[k][p] = c * up - s * uq;
                    U[k][q] = s * up + c * uq;
                }
            }
    }
    int idx[3] = {0, 1, 2};
    double d[3] = {a[0][0], a[1][1], a[2][2]};
    for (int i = 0; i < 2; ++i)                        /* ascending */
        for (int j = 0; j < 2 - i; ++j)
            if (d[idx[j]] > d[idx[j + 1]]) { int t = idx[j]; idx[j] = idx[j + 1]; idx[j + 1] = t; }
    for (int i = 0; i < 3; ++i) {
        lam[i] = d[idx[i]];
        if (V)
            for (int k = 0; k < 3; ++k) V[k][i] = U[k][idx[i]];
    }
}

static void jacobi3(const double Hin[3][3], double lam[3]) { jacobi3v(Hin, lam, NULL); }

void orc_eig3(const double* h6, double* lam) {
    double H[3][3] = {{h6[0], h6[1], h6[2]}, {h6[1], h6[3], h6[4]}, {h6[2], h6[4], h6[5]}};
    jacobi3(H, lam);
}

/* Eq. radiusAniso3D with the largest |eigenvalue| (isotropic records, Sec. 6) */
double orc_radius(double LY, const double* h6, double eps, double r_min, double r_max, int* status, double* lam) {
    orc_eig3(h6, lam);
    double lmax = fmax(fabs(lam[0]), fmax(fabs(lam[1]), fabs(lam[2])));
    if (!isfinite(LY) || !isfinite(lmax)) { *status |= REC_NONFINITE | REC_CLAMP_LO; return r_min; }
    if (!(LY > 0)) { *status |= REC_CLAMP_LO; return r_min; }
    if (lmax == 0.0) { *status |= REC_CLAMP_HI; return r_max; }
    double R = pow(15.0 * LY * eps / (4.0 * ORC_PI * lmax), 0.2);
    if (R < r_min) { *status |= REC_CLAMP_LO; return r_min; }
    if (R > r_max) { *status |= REC_CLAMP_HI; return r_max; }
    return R;
}

static const double LUM[3] = {0.2126, 0.7152, 0.0722};   /* Rec.709 luminance */

/* Ellipsoidal records (Eq. radiusAniso3D per eigenvalue, Sec. 5 and supplemental S.11):
 * principal radius R_i = (15 L_Y eps / (4 pi |lambda_i|))^(1/5) along the eigenvector v_i
 * of the luminance Hessian, clamped to [r_min, r_max] like the isotropic radius (L_Y <= 0
 * or non-finite: r_min on every axis; lambda_i = 0: r_max on that axis).  Outputs:
 * lam[3] ascending, radii[3] in that order, axes[9] row i = v_i, metric[6] = the
 * symmetric M = sum_i v_i v_i^T / R_i^2 (upper triangle xx xy xz yy yz zz), so that the
 * record's region is D^T M D < 1. */
int orc_aniso(double LY, const double* h6, double eps, double r_min, double r_max, double* lam, double* radii,
              double* axes, double* metric) {
    double H[3][3] = {{h6[0], h6[1], h6[2]}, {h6[1], h6[3], h6[4]}, {h6[2], h6[4], h6[5]}};
    double V[3][3];
    jacobi3v(H, lam, V);
    int status = 0;
    int bad = !isfinite(LY) || !isfinite(lam[0]) || !isfinite(lam[1]) || !isfinite(lam[2]);
    for (int i = 0; i < 3; ++i) {
        double R;
        double al = fabs(lam[i]);
        if (bad) { status |= REC_NONFINITE | REC_CLAMP_LO; R = r_min; }
        else if (!(LY > 0)) { status |= REC_CLAMP_LO; R = r_min; }
        else if (al == 0.0) { status |= REC_CLAMP_HI; R = r_max; }
        else {
            R = pow(15.0 * LY * eps / (4.0 * ORC_PI * al), 0.2);
            if (R < r_min) { status |= REC_CLAMP_LO; R = r_min; }
            if (R > r_max) { status |= REC_CLAMP_HI; R = r_max; }
        }
        radii[i] = R;
        for (int k = 0; k < 3; ++k) axes[3 * i + k] = V[k][i];
    }
    static const int IJ[6][2] = {{0, 0}, {0, 1}, {0, 2}, {1, 1}, {1, 2}, {2, 2}};
    for (int e = 0; e < 6; ++e) {
        double m = 0.0;
        for (int i = 0; i < 3; ++i) m += V[IJ[e][0]][i] * V[IJ[e][1]][i] / (radii[i] * radii[i]);
        metric[e] = m;
    }
    return status;
}

/* ---------------------------------------------------- one record (Secs. 4-5) */
typedef struct {
    int nb, ns, V, N, K;
    int replay;        /* 1: primary hits were given (no primary decision is uncertain) */
    int full;          /* 1: ray ends and visibility were given too (no decision is uncertain) */
    double* t_key;     /* [V] the parameter that decides clamps and furthest vertices */
    int n_lit_replayed, n_unexplained;
    v3 x;
    v3* dir;
    double* t_end;
    int* hit;
    double* Lo_surf;   /* [V][3] */
    double* Lo_med;    /* [K][V][3] */
    /* shadow-ray decisions near a tie: |change| summed over lights, signed change, count */
    double* dLo_surf;  /* [V][3] */
    double* sLo_surf;  /* [V][3] */
    int* nsh_surf;     /* [V] */
    double* dLo_med;   /* [K][V][3] */
    double* sLo_med;   /* [K][V][3] */
    int* nsh_med;      /* [K][V] */
    unsigned char* unc_clamp;   /* [K][V] clamp decision (t_k against the ray's end) near a tie */
    double* calt_Lo_med;        /* [K][V][3] radiance of the unclamped alternative of a clamped vertex */
    unsigned char* unc_prim;    /* [V] primary hit near a tie */
    double* margin_e;  /* per primary ray: edge margin */
    double* tie;
    double* t_unc;     /* [V] relative uncertainty of t_end: TIE_T (1 + 1/|cos incidence|) */
    int n_replayed;    /* rays whose given hit differs from the oracle's own */
    int n_bad_replay;  /* given hit ids out of range (ignored) */
    /* the other outcome of a near-tie primary ray (found by re-tracing perturbed directions) */
    double* alt_t;     /* [V] */
    int* alt_hit;      /* [V] */
    double* alt_Lo_surf;   /* [V][3] */
    double* alt_Lo_med;    /* [K][V][3] medium radiance where the alternative ray is unclamped */
} shells_t;

static void shells_free(shells_t* S) {
    free(S->dir); free(S->t_end); free(S->hit); free(S->Lo_surf); free(S->Lo_med);
    free(S->dLo_surf); free(S->sLo_surf); free(S->nsh_surf);
    free(S->dLo_med); free(S->sLo_med); free(S->nsh_med);
    free(S->unc_clamp); free(S->calt_Lo_med); free(S->unc_prim);
    free(S->margin_e); free(S->tie); free(S->t_unc); free(S->t_key);
    free(S->alt_t); free(S->alt_hit); free(S->alt_Lo_surf); free(S->alt_Lo_med);
}

/* plane parameter of the ray (x, d) on triangle id, ignoring its edges (replayed hits) */
static int plane_t(const orc_scene* s, int id, v3 x, v3 d, double* t) {
    otri T;
    T.a = ldv(s->in.tri_v + 9 * id);
    T.b = ldv(s->in.tri_v + 9 * id + 3);
    T.c = ldv(s->in.tri_v + 9 * id + 6);
    double u, v;
    return mt(x, d, &T, t, &u, &v) && *t > 0.0;
}

/* trace the ray set, the shells and every vertex radiance (Sec. 4, Sec. 6 Implementation).
 * replay (nullable): a primary hit id per ray (-1 = no hit) to use instead of the oracle's
 * own closest hit (reading R16's replay: the reduction is then compared on the same hits). */
static int lit_bit(const orc_replay* R, int k, int v) {
    if (k >= R->shells) return 0;
    int words = (R->stride + 31) / 32;
    return (int)((R->lit[(size_t)k * words + (size_t)(v >> 5)] >> (v & 31)) & 1u);
}

/* shell k's parameter t_k as the kernel computes it in FP32 */
static float tk_f32(int k, float dt) {
    float a = (float)k - 0.5f;
    return a * dt;
}

/* vertex v of shell k >= 1 is open (t_k before its ray's end): FP64, or the given FP32 ends */
static int vertex_open(const shells_t* S, const orc_params* p, int k, int v) {
    if (S->full) return tk_f32(k, p->dt) < (float)S->t_key[v];
    return ((double)k - 0.5) * (double)p->dt < S->t_end[v];
}

/* a given visibility decision: take the other shadow outcome where it is a near tie */
static void replay_lit(shells_t* S, int given, double Lo[3], const double sLo[3], int nsh) {
    int lit = Lo[0] != 0.0 || Lo[1] != 0.0 || Lo[2] != 0.0;
    if (given == lit) return;
    if (nsh == 1) {
        for (int c = 0; c < 3; ++c) Lo[c] += sLo[c];
        S->n_lit_replayed++;
    } else {
        S->n_unexplained++;
    }
}

static void build_shells(const orc_scene* s, v3 x, const orc_params* p, int nb, int ns, int64_t rec,
                         const orc_replay* R, shells_t* S) {
    memset(S, 0, sizeof(*S));
    S->nb = nb; S->ns = ns; S->N = nb * ns; S->V = S->N + 2; S->x = x;
    const int32_t* replay = R ? R->hit : NULL;
    S->replay = replay != NULL;
    S->full = R && R->t && R->lit;
    int V = S->V, track = p->track_margins || S->full;
    S->t_key = (double*)malloc(sizeof(double) * V);
    S->dir = (v3*)malloc(sizeof(v3) * V);
    S->t_end = (double*)malloc(sizeof(double) * V);
    S->hit = (int*)malloc(sizeof(int) * V);
    S->Lo_surf = (double*)calloc((size_t)V * 3, sizeof(double));
    S->dLo_surf = (double*)calloc((size_t)V * 3, sizeof(double));
    S->sLo_surf = (double*)calloc((size_t)V * 3, sizeof(double));
    S->nsh_surf = (int*)calloc((size_t)V, sizeof(int));
    S->unc_prim = (unsigned char*)calloc((size_t)V, 1);
    S->margin_e = (double*)malloc(sizeof(double) * V);
    S->tie = (double*)malloc(sizeof(double) * V);
    S->t_unc = (double*)malloc(sizeof(double) * V);
    S->alt_t = (double*)malloc(sizeof(double) * V);
    S->alt_hit = (int*)malloc(sizeof(int) * V);
    S->alt_Lo_surf = (double*)calloc((size_t)V * 3, sizeof(double));
    double tmax = 0.0;
    for (int v = 0; v < V; ++v) {
        v3 d = ray_direction(p, nb, ns, rec, v);
        S->dir[v] = d;
        S->margin_e[v] = INFINITY;
        S->tie[v] = INFINITY;
        double t;
        int id;
        if (s->in.sphere_mode) {
            v3 oc = sub(x, ldv(s->in.sphere_c));
            double bq = dot(d, oc), cq = dot(oc, oc) - (double)s->in.sphere_r * (double)s->in.sphere_r;
            t = -bq + sqrt(bq * bq - cq);
            id = 0;
        } else {
            double tie_val = INFINITY;
            id = closest_hit(s, x, d, &t, &S->margin_e[v], &S->tie[v], &tie_val, track);
            if (track && (S->margin_e[v] < TIE_EDGE || tie_val < TIE_T)) S->unc_prim[v] = 1;
            if (replay) {
                int rid = replay[v];
                double tr;
                if (rid < -1 || rid >= s->n || (rid >= 0 && !plane_t(s, rid, x, d, &tr))) {
                    S->n_bad_replay++;                 /* keep the oracle's own hit */
                } else if (rid != id) {
                    S->n_replayed++;
                    id = rid;
                    if (rid >= 0) t = tr;
                }
                S->unc_prim[v] = 0;                    /* the decision is the given one */
            }
        }
        double cinc = 1.0;                           /* |cos| between the ray and the surface it ends on */
        if (id >= 0 && !s->in.sphere_mode) {
            v3 a = ldv(s->in.tri_v + 9 * id), b = ldv(s->in.tri_v + 9 * id + 3), c = ldv(s->in.tri_v + 9 * id + 6);
            v3 n = cross(sub(b, a), sub(c, a));
            cinc = fabs(dot(n, d)) / norm(n);
        } else if (id < 0) {
            cinc = fmax(fabs(d.x), fmax(fabs(d.y), fabs(d.z)));  /* lower bound over the exit face */
            double te = cube_exit(x, d);
            for (int k = 0; k < 3; ++k) {                         /* the axis that sets the exit */
                double xk = comp(x, k), dk = comp(d, k);
                double tk = dk > 0 ? (1.0 - xk) / dk : (dk < 0 ? -xk / dk : INFINITY);
                if (tk == te) cinc = fabs(dk);
            }
        }
        S->t_unc[v] = TIE_T * (1.0 + 1.0 / fmax(cinc, 1e-6));
        if (id >= 0) {
            S->t_end[v] = t;
            S->hit[v] = id;
            v3 y = add(x, scl(d, t));
            if (s->in.sphere_mode) {
                for (int c = 0; c < 3; ++c) S->Lo_surf[3 * v + c] = (double)s->in.sphere_Le[c];
            } else {
                surface_radiance(s, id, y, d, &S->Lo_surf[3 * v], &S->dLo_surf[3 * v], &S->sLo_surf[3 * v],
                                 &S->nsh_surf[v], track);
            }
        } else {
            S->t_end[v] = cube_exit(x, d);
            S->hit[v] = -1;
        }
        S->t_key[v] = S->t_end[v];
        if (S->full) {
            double tg = (double)R->t[v];
            S->t_key[v] = tg;
            if (fabs(tg - S->t_end[v]) > fmax(4.0 * S->t_unc[v] * S->t_end[v], 1e-6)) S->n_unexplained++;
            if (tg > tmax) tmax = tg;
            replay_lit(S, lit_bit(R, 0, v), &S->Lo_surf[3 * v], &S->sLo_surf[3 * v], S->nsh_surf[v]);
        }
        S->alt_t[v] = S->t_end[v];
        S->alt_hit[v] = S->hit[v];
        if (S->unc_prim[v]) {
            /* the outcome a slightly different ray would see: re-trace directions turned by
             * 1e-4 rad about two axes normal to d; keep the one that differs most */
            v3 e1 = fabs(d.x) < 0.9 ? cross(d, mk(1, 0, 0)) : cross(d, mk(0, 1, 0));
            e1 = scl(e1, 1.0 / norm(e1));
            v3 e2 = cross(d, e1);
            double best = -1.0;
            for (int q = 0; q < 4; ++q) {
                v3 dq = add(d, scl(q < 2 ? e1 : e2, (q & 1) ? -1e-4 : 1e-4));
                dq = scl(dq, 1.0 / norm(dq));
                double tq, m0 = INFINITY, m1 = INFINITY, m2 = INFINITY;
                int iq = closest_hit(s, x, dq, &tq, &m0, &m1, &m2, 0);
                if (iq < 0) tq = cube_exit(x, d);
                double diff = fabs(tq - S->t_end[v]) + (iq != S->hit[v] ? 1e-12 : 0.0);
                if (iq != S->hit[v] && !(iq >= 0 && S->hit[v] >= 0 && same_surface(s, iq, S->hit[v])) && diff > best) {
                    best = diff;
                    S->alt_t[v] = tq;
                    S->alt_hit[v] = iq;
                }
            }
            if (S->alt_hit[v] >= 0 && S->alt_hit[v] != S->hit[v])
                surface_radiance(s, S->alt_hit[v], add(x, scl(d, S->alt_t[v])), d, &S->alt_Lo_surf[3 * v], NULL, NULL,
                                 NULL, 0);
            if (S->alt_t[v] > tmax) tmax = S->alt_t[v];
        }
        if (S->t_end[v] > tmax) tmax = S->t_end[v];
    }
    double dt = (double)p->dt;
    S->K = p->surface_only ? 0 : (int)ceil(tmax / dt) + (S->full ? 1 : 0);
    size_t KV = (size_t)(S->K > 0 ? S->K : 1) * V;
    S->Lo_med = (double*)calloc(KV * 3, sizeof(double));
    S->dLo_med = (double*)calloc(KV * 3, sizeof(double));
    S->sLo_med = (double*)calloc(KV * 3, sizeof(double));
    S->nsh_med = (int*)calloc(KV, sizeof(int));
    S->unc_clamp = (unsigned char*)calloc(KV, 1);
    S->calt_Lo_med = (double*)calloc(KV * 3, sizeof(double));
    S->alt_Lo_med = (double*)calloc(KV * 3, sizeof(double));
    for (int k = 1; k <= S->K; ++k) {
        double tk = ((double)k - 0.5) * dt;
        for (int v = 0; v < V; ++v) {
            size_t o = (size_t)(k - 1) * V + v;
            v3 y = add(x, scl(S->dir[v], tk));
            int near = track && fabs(tk - S->t_end[v]) < S->t_unc[v] * S->t_end[v];
            int open = vertex_open(S, p, k, v);
            if (open)
                medium_radiance(s, y, S->dir[v], &S->Lo_med[3 * o], &S->dLo_med[3 * o], &S->sLo_med[3 * o],
                                &S->nsh_med[o], track);
            else if (near)      /* clamped now; the alternative is an unclamped medium vertex at t_k */
                medium_radiance(s, y, S->dir[v], &S->calt_Lo_med[3 * o], NULL, NULL, NULL, 0);
            if (near) S->unc_clamp[o] = 1;
            if (S->full) {
                if (open) replay_lit(S, lit_bit(R, k, v), &S->Lo_med[3 * o], &S->sLo_med[3 * o], S->nsh_med[o]);
                else if (lit_bit(R, k, v)) S->n_unexplained++;     /* given lit, but clamped here */
                if (open != (tk < S->t_end[v]) && !near) S->n_unexplained++;
            }
            if (S->unc_prim[v] && tk < S->alt_t[v]) {
                if (tk < S->t_end[v]) memcpy(&S->alt_Lo_med[3 * o], &S->Lo_med[3 * o], 3 * sizeof(double));
                else medium_radiance(s, y, S->dir[v], &S->alt_Lo_med[3 * o], NULL, NULL, NULL, 0);
            }
        }
    }
}

/* The discrete decisions of one vertex that FP32 may take the other way: its primary ray's
 * hit (ALT_PRIM), its clamp at the ray's end (ALT_CLAMP, medium shells), its shadow ray
 * (ALT_SHADOW, one light near a tie). */
enum { ALT_SHADOW = 1, ALT_CLAMP = 2, ALT_PRIM = 4 };

/* vertex v of shell k (k = 0 surface shell, k >= 1 medium shell) with the decisions in
 * `alts` taken the other way: its ray parameter (returned), radiance, the relative
 * uncertainty of that parameter's comparison with other vertices', and *open = 1 for an
 * unclamped medium vertex (every such vertex of a shell sits at the same t_k, in any
 * precision, and a clamped one at its ray's end t_end <= t_k) */
static double vertex_state(const shells_t* S, const orc_params* p, int k, int v, int alts, double Lo[3],
                           double* t_tol, int* open) {
    Lo[0] = Lo[1] = Lo[2] = 0.0;
    *t_tol = S->t_unc[v] + 2.0 * TIE_T;
    *open = 0;
    if (k == 0) {
        if (alts & ALT_PRIM) {
            if (S->alt_hit[v] >= 0) memcpy(Lo, &S->alt_Lo_surf[3 * v], 3 * sizeof(double));
            return S->alt_t[v];
        }
        if (S->hit[v] >= 0) {
            memcpy(Lo, &S->Lo_surf[3 * v], 3 * sizeof(double));
            if (alts & ALT_SHADOW)
                for (int c = 0; c < 3; ++c) Lo[c] += S->sLo_surf[3 * v + c];
        }
        return S->t_end[v];
    }
    size_t o = (size_t)(k - 1) * S->V + v;
    double tk = ((double)k - 0.5) * (double)p->dt;
    if (alts & ALT_PRIM) {
        if (tk < S->alt_t[v]) {
            memcpy(Lo, &S->alt_Lo_med[3 * o], 3 * sizeof(double));
            *t_tol = 2.0 * TIE_T;
            *open = 1;
            return tk;
        }
        return S->alt_t[v];
    }
    int unclamped = tk < S->t_end[v];
    if (alts & ALT_CLAMP) {
        if (unclamped) return tk;                    /* clamped instead: zero-radiance sample at t_end <= t_k */
        memcpy(Lo, &S->calt_Lo_med[3 * o], 3 * sizeof(double));
        *t_tol = 2.0 * TIE_T;
        *open = 1;
        return tk;
    }
    if (!unclamped) return S->t_end[v];              /* zero-radiance sample at the occluder (Sec. 4) */
    memcpy(Lo, &S->Lo_med[3 * o], 3 * sizeof(double));
    if (alts & ALT_SHADOW)
        for (int c = 0; c < 3; ++c) Lo[c] += S->sLo_med[3 * o + c];
    *t_tol = 2.0 * TIE_T;
    *open = 1;
    return tk;
}

/* a furthest-vertex set that rounding can produce: nonempty, within the near-furthest
 * vertices, and holding every open vertex of a medium-shell cell (they share t_k, and a
 * clamped vertex never lies beyond it) */
static int far_set_valid(int fs, int nearm, int openm) {
    if (fs == 0 || (fs & nearm) != fs) return 0;
    return (fs & openm) == openm;
}

static int far_set_ambiguous(int nearm, int openm) {
    if (openm) return (nearm & ~openm) != 0;
    return (nearm & (nearm - 1)) != 0;               /* two or more near-furthest vertices */
}

/* vertex v of shell k as computed: ray parameter (returned), radiance, and the parameter
 * that orders it against the cell's other vertices (the same, or in full replay the FP32
 * value the decisions were taken on) */
static double vertex_t(const shells_t* S, const orc_params* p, int k, int v, const double** Lo, double* key) {
    static const double zero[3] = {0, 0, 0};
    if (k == 0) {
        *Lo = S->hit[v] >= 0 ? &S->Lo_surf[3 * v] : zero;
        *key = S->t_key[v];
        return S->t_end[v];
    }
    size_t o = (size_t)(k - 1) * S->V + v;
    double tk = ((double)k - 0.5) * (double)p->dt;
    if (vertex_open(S, p, k, v)) {
        *Lo = &S->Lo_med[3 * o];
        *key = S->full ? (double)tk_f32(k, p->dt) : tk;
        return tk;
    }
    *Lo = zero;                                      /* zero-radiance sample at the occluder (Sec. 4) */
    *key = S->t_key[v];
    return S->t_end[v];
}

/* the change one decision makes to the record, summed (as vectors) over the cells it touches */
typedef struct {
    int kind, k, v;
    double L[3], g[3][3], H[3][3][3];
} decision_t;

typedef struct {
    double L[3], g[3][3], H[3][3][3];
    double sumHnorm;   /* sum of per-cell luminance Hessian Frobenius norms */
    int n_degen;
    double bud_L[3], bud_g[3], bud_H[3];
    int n_unc;
    decision_t* dec;   /* decisions whose cells each hold no other uncertain decision */
    int n_dec, cap_dec;
} ffsum;

static decision_t* find_decision(ffsum* acc, int kind, int k, int v) {
    for (int i = 0; i < acc->n_dec; ++i)
        if (acc->dec[i].kind == kind && acc->dec[i].k == k && acc->dec[i].v == v) return &acc->dec[i];
    if (acc->n_dec == acc->cap_dec) {
        acc->cap_dec = acc->cap_dec ? 2 * acc->cap_dec : 16;
        acc->dec = (decision_t*)realloc(acc->dec, sizeof(decision_t) * (size_t)acc->cap_dec);
    }
    decision_t* d = &acc->dec[acc->n_dec++];
    memset(d, 0, sizeof(*d));
    d->kind = kind; d->k = k; d->v = v;
    return d;
}

/* lo_grad: the light's propagation direction at medium vertex v of shell k (position y)
 * and the HG phase toward the record centre, where the vertex radiance was computed (the
 * direction to the centre is -d_v).  Returns 0 (constant L_o) for surface vertices, closed
 * vertices and when lo_grad is off. */
static int vertex_light(const orc_scene* s, const shells_t* S, const orc_params* p, int k, int v, int open, v3 y,
                        v3* lp, double* f0) {
    *f0 = 0.0;
    if (!p->lo_grad || k == 0 || !open || s->in.n_lights != 1) return 0;
    v3 l = sub(y, ldv(s->in.light_pos));
    *lp = scl(l, 1.0 / norm(l));
    *f0 = orc_hg(-dot(*lp, S->dir[v]), (double)s->in.g);
    return 1;
}

/* One cell of shell k with the decisions alts[q] of its vertices taken the other way.
 * far_set (bit mask) overrides the furthest vertices when nonzero.  Fills *co (zero for a
 * dark or degenerate cell) and *near_set: the vertices whose parameter is within FP32
 * rounding of the largest, any nonempty subset of which FP32 may take as the furthest. */
static int eval_cell(const orc_scene* s, const shells_t* S, const orc_params* p, v3 x_eval, int k, const int vi[3],
                     const int alts[3], int far_set, double weight, cellout* co, int* near_set, int* open_set) {
    double Lo[3][3], t[3], tol[3];
    int op[3];
    v3 y[3];
    for (int q = 0; q < 3; ++q) {
        t[q] = vertex_state(S, p, k, vi[q], alts[q], Lo[q], &tol[q], &op[q]);
        y[q] = add(S->x, scl(S->dir[vi[q]], t[q]));
    }
    double tmx = fmax(t[0], fmax(t[1], t[2]));
    int canon = 0, nearm = 0, openm = 0;
    for (int q = 0; q < 3; ++q) {
        if (t[q] == tmx) canon |= 1 << q;
        if (tmx - t[q] <= tol[q] * tmx) nearm |= 1 << q;
        if (op[q]) openm |= 1 << q;
    }
    if (near_set) *near_set = nearm;
    if (open_set) *open_set = openm;
    int fs = far_set ? far_set : canon;
    v3 yf[3], lpf[3];
    double f0f[3];
    const double* Lf[3];
    int nf = 0, dark = 1;
    for (int q = 0; q < 3; ++q)
        if (fs & (1 << q)) {
            yf[nf] = y[q]; Lf[nf] = Lo[q];
            vertex_light(s, S, p, k, vi[q], op[q], y[q], &lpf[nf], &f0f[nf]);
            ++nf;
            if (Lo[q][0] != 0.0 || Lo[q][1] != 0.0 || Lo[q][2] != 0.0) dark = 0;
        }
    memset(co, 0, sizeof(*co));
    if (dark) return 1;
    v3 wo = ldv(p->omega_o);
    int ok = cell_radiance(x_eval, y[0], y[1], y[2], nf, yf, Lf, s->sigma_t, (double)s->in.g, wo, weight,
                           p->general_derivs, p->ff_signed, co, lpf, f0f);
    if (!ok) memset(co, 0, sizeof(*co));
    return ok;
}

static void cell_diff_norms(const cellout* a, const cellout* b, double nL[3], double ng[3], double nH[3]) {
    for (int ch = 0; ch < 3; ++ch) {
        double gn = 0, hn = 0;
        for (int i = 0; i < 3; ++i) {
            double dg = a->g[ch][i] - b->g[ch][i];
            gn += dg * dg;
            for (int j = 0; j < 3; ++j) {
                double dh = a->H[ch][i][j] - b->H[ch][i][j];
                hn += dh * dh;
            }
        }
        nL[ch] = fabs(a->L[ch] - b->L[ch]);
        ng[ch] = sqrt(gn);
        nH[ch] = sqrt(hn);
    }
}

/* Decision budget of one cell (track_margins).  The record's change under any set of
 * flipped decisions is the sum over cells of each cell's change.  A cell touched by exactly
 * one binary decision, with an unambiguous furthest-vertex set both ways, changes by that
 * decision's exact difference: it is added (as a vector) to the decision's total, whose
 * norm enters the budget once.  Any other cell (several decisions, an ambiguous furthest
 * set, several lights near a tie at one vertex) adds the largest change over every
 * combination of its decisions and furthest sets.  The budget therefore bounds the change
 * of every combination, and equals it when a single decision flips. */
static void cell_budget(const orc_scene* s, const shells_t* S, const orc_params* p, v3 x_eval, int k, int c,
                        const int vi[3], double weight, ffsum* acc) {
    int dq[12], dk[12];
    int nd = 0, multi = 0;
    for (int q = 0; q < 3; ++q) {
        int v = vi[q];
        if (!S->replay && S->unc_prim[v]) { dq[nd] = q; dk[nd] = ALT_PRIM; ++nd; }
        int nsh;
        if (k == 0) nsh = S->hit[v] >= 0 ? S->nsh_surf[v] : 0;
        else {
            size_t o = (size_t)(k - 1) * S->V + v;
            double tk = ((double)k - 0.5) * (double)p->dt;
            nsh = tk < S->t_end[v] ? S->nsh_med[o] : 0;
            if (S->unc_clamp[o]) { dq[nd] = q; dk[nd] = ALT_CLAMP; ++nd; }
        }
        if (nsh == 1) { dq[nd] = q; dk[nd] = ALT_SHADOW; ++nd; }
        else if (nsh > 1) multi = 1;
    }
    static const int none[3] = {0, 0, 0};
    cellout cur;
    int near_cur, open_cur;
    eval_cell(s, S, p, x_eval, k, vi, none, 0, weight, &cur, &near_cur, &open_cur);
    int amb_cur = far_set_ambiguous(near_cur, open_cur);
    if (nd == 0 && !amb_cur && !multi) return;
    acc->n_unc++;
    if (nd == 1 && !amb_cur && !multi) {
        int alts[3] = {0, 0, 0};
        alts[dq[0]] = dk[0];
        cellout alt;
        int near_alt, open_alt;
        eval_cell(s, S, p, x_eval, k, vi, alts, 0, weight, &alt, &near_alt, &open_alt);
        if (!far_set_ambiguous(near_alt, open_alt)) {
            decision_t* d = find_decision(acc, dk[0], dk[0] == ALT_PRIM ? -1 : k, vi[dq[0]]);
            for (int ch = 0; ch < 3; ++ch) {
                d->L[ch] += alt.L[ch] - cur.L[ch];
                for (int i = 0; i < 3; ++i) {
                    d->g[ch][i] += alt.g[ch][i] - cur.g[ch][i];
                    for (int j = 0; j < 3; ++j) d->H[ch][i][j] += alt.H[ch][i][j] - cur.H[ch][i][j];
                }
            }
            return;
        }
    }
    /* every combination of the cell's decisions and of its furthest sets */
    double mL[3] = {0, 0, 0}, mg[3] = {0, 0, 0}, mH[3] = {0, 0, 0};
    for (int combo = 0; combo < (1 << nd); ++combo) {
        int alts[3] = {0, 0, 0};
        for (int i = 0; i < nd; ++i)
            if (combo & (1 << i)) alts[dq[i]] |= dk[i];
        int nearm, openm;
        cellout co;
        eval_cell(s, S, p, x_eval, k, vi, alts, 0, weight, &co, &nearm, &openm);
        for (int fs = 1; fs < 8; ++fs) {           /* every furthest set rounding can produce */
            if (!far_set_valid(fs, nearm, openm)) continue;
            eval_cell(s, S, p, x_eval, k, vi, alts, fs, weight, &co, NULL, NULL);
            double nL[3], ng[3], nH[3];
            cell_diff_norms(&co, &cur, nL, ng, nH);
            for (int ch = 0; ch < 3; ++ch) {
                mL[ch] = fmax(mL[ch], nL[ch]);
                mg[ch] = fmax(mg[ch], ng[ch]);
                mH[ch] = fmax(mH[ch], nH[ch]);
            }
        }
    }
    if (multi) {
        /* several lights near a tie at one vertex: bound the change of its radiance by the
         * sum of those lights' terms, carried by the furthest vertex */
        double U[3] = {0, 0, 0};
        for (int q = 0; q < 3; ++q) {
            const double* dl;
            if (k == 0) dl = &S->dLo_surf[3 * vi[q]];
            else dl = &S->dLo_med[3 * ((size_t)(k - 1) * S->V + vi[q])];
            for (int ch = 0; ch < 3; ++ch) U[ch] += dl[ch];
        }
        double Lo_dummy[3], tol, tq[3];
        int opq;
        v3 y[3];
        for (int q = 0; q < 3; ++q) {
            tq[q] = vertex_state(S, p, k, vi[q], 0, Lo_dummy, &tol, &opq);
            y[q] = add(S->x, scl(S->dir[vi[q]], tq[q]));
        }
        int qf = tq[0] >= tq[1] && tq[0] >= tq[2] ? 0 : (tq[1] >= tq[2] ? 1 : 2);
        v3 yf = y[qf];
        const double* Up[1] = {U};
        cellout cu;
        v3 wo = ldv(p->omega_o);
        if (cell_radiance(x_eval, y[0], y[1], y[2], 1, &yf, Up, s->sigma_t, (double)s->in.g, wo, weight,
                          p->general_derivs, p->ff_signed, &cu, NULL, NULL)) {
            static const cellout zero_cell;
            double nL[3], ng[3], nH[3];
            cell_diff_norms(&cu, &zero_cell, nL, ng, nH);
            for (int ch = 0; ch < 3; ++ch) { mL[ch] += nL[ch]; mg[ch] += ng[ch]; mH[ch] += nH[ch]; }
        }
    }
    (void)c;
    for (int ch = 0; ch < 3; ++ch) {
        acc->bud_L[ch] += mL[ch];
        acc->bud_g[ch] += mg[ch];
        acc->bud_H[ch] += mH[ch];
    }
}

/* Eqs. ApprxRadiance, SegmentRadianceGradient, SegmentRadianceHessian over a range of
 * shells, evaluated at x_eval with the vertices and furthest-vertex choices of S frozen */
static void ff_accumulate(const orc_scene* s, const shells_t* S, const orc_params* p, v3 x_eval, int k0, int k1,
                          ffsum* acc) {
    memset(acc, 0, sizeof(*acc));
    int ncell = 2 * S->N;
    v3 wo = ldv(p->omega_o);
    for (int k = k0; k <= k1; ++k) {
        double weight = (k == 0) ? 1.0 : (double)s->in.sigma_s * (double)p->dt;   /* 1 / pdf(ring) */
        for (int c = 0; c < ncell; ++c) {
            int vi[3];
            cell_vertices(S->nb, S->ns, c, &vi[0], &vi[1], &vi[2]);
            const double* Lo[3];
            double t[3], key[3];
            v3 y[3];
            for (int q = 0; q < 3; ++q) {
                t[q] = vertex_t(S, p, k, vi[q], &Lo[q], &key[q]);
                y[q] = add(S->x, scl(S->dir[vi[q]], t[q]));
            }
            /* furthest vertices (R9): all vertices at the largest t */
            double tmx = fmax(key[0], fmax(key[1], key[2]));
            int nf = 0;
            v3 yf[3], lpf[3];
            double f0f[3];
            const double* Lf[3];
            for (int q = 0; q < 3; ++q)
                if (key[q] == tmx) {
                    yf[nf] = y[q]; Lf[nf] = Lo[q];
                    vertex_light(s, S, p, k, vi[q], k > 0 && vertex_open(S, p, k, vi[q]), y[q], &lpf[nf], &f0f[nf]);
                    ++nf;
                }
            if (p->track_margins && !S->full) cell_budget(s, S, p, x_eval, k, c, vi, weight, acc);
            int dark = 1;
            for (int q = 0; q < nf; ++q)
                if (Lf[q][0] != 0.0 || Lf[q][1] != 0.0 || Lf[q][2] != 0.0) dark = 0;
            if (dark) continue;
            cellout co;
            int ok = cell_radiance(x_eval, y[0], y[1], y[2], nf, yf, Lf, s->sigma_t, (double)s->in.g, wo, weight,
                                   p->general_derivs, p->ff_signed, &co, lpf, f0f);
            if (!ok) { acc->n_degen++; continue; }
            double hn = 0.0;
            for (int i = 0; i < 3; ++i)
                for (int j = 0; j < 3; ++j) {
                    double hy = LUM[0] * co.H[0][i][j] + LUM[1] * co.H[1][i][j] + LUM[2] * co.H[2][i][j];
                    hn += hy * hy;
                }
            acc->sumHnorm += sqrt(hn);
            for (int ch = 0; ch < 3; ++ch) {
                acc->L[ch] += co.L[ch];
                for (int i = 0; i < 3; ++i) acc->g[ch][i] += co.g[ch][i];
                for (int i = 0; i < 3; ++i)
                    for (int j = 0; j < 3; ++j) acc->H[ch][i][j] += co.H[ch][i][j];
            }
        }
    }
    /* each decision's total change enters the budget once */
    for (int i = 0; i < acc->n_dec; ++i) {
        const decision_t* d = &acc->dec[i];
        for (int ch = 0; ch < 3; ++ch) {
            double gn = 0, hn = 0;
            for (int a = 0; a < 3; ++a) {
                gn += d->g[ch][a] * d->g[ch][a];
                for (int b = 0; b < 3; ++b) hn += d->H[ch][a][b] * d->H[ch][a][b];
            }
            acc->bud_L[ch] += fabs(d->L[ch]);
            acc->bud_g[ch] += sqrt(gn);
            acc->bud_H[ch] += sqrt(hn);
        }
    }
    free(acc->dec);
    acc->dec = NULL;
    acc->n_dec = acc->cap_dec = 0;
}

static void pack_h6(const double H[3][3], double* o) {
    o[0] = H[0][0]; o[1] = H[0][1]; o[2] = H[0][2]; o[3] = H[1][1]; o[4] = H[1][2]; o[5] = H[2][2];
}

static void compute_record(const orc_scene* s, const orc_params* p, v3 x, int nb, int ns, int64_t rec,
                           const orc_replay* replay, double* out, int32_t* dbg_hit, double* dbg_t, double* dbg_margin,
                           double* dbg_tie, uint32_t* dbg_lit, int dbg_shells, int dbg_stride) {
    memset(out, 0, sizeof(double) * ORC_OUT_STRIDE);
    shells_t S;
    build_shells(s, x, p, nb, ns, rec, replay, &S);
    const int bud_on = !S.full;           /* in full replay every decision is the given one */
    /* Monte Carlo radiance (Eqs. outLF, mediaLFin, curveLFin with equal-solid-angle strata) */
    v3 wo = ldv(p->omega_o);
    double dt = (double)p->dt, st = s->sigma_t, ss = (double)s->in.sigma_s;
    double Lss[3] = {0, 0, 0}, Lms[3] = {0, 0, 0}, bud[3] = {0, 0, 0};
    for (int v = 0; v < S.N; ++v) {
        v3 d = S.dir[v];
        double f = orc_hg(dot(scl(d, -1.0), wo), (double)s->in.g);   /* w_i = -d */
        double w = 4.0 * ORC_PI / (double)S.N * f;
        if (S.hit[v] >= 0) {
            double T = exp(-st * S.t_end[v]);
            for (int c = 0; c < 3; ++c) {
                Lss[c] += w * T * S.Lo_surf[3 * v + c];
                if (bud_on) bud[c] += w * T * S.dLo_surf[3 * v + c];
            }
        }
        for (int k = 1; k <= S.K; ++k) {
            double tk = ((double)k - 0.5) * dt;
            size_t o = (size_t)(k - 1) * S.V + v;
            double T = exp(-st * tk);
            if (vertex_open(&S, p, k, v))
                for (int c = 0; c < 3; ++c) Lms[c] += w * ss * dt * T * S.Lo_med[3 * o + c];
            if (!bud_on) continue;
            for (int c = 0; c < 3; ++c) bud[c] += w * ss * dt * T * S.dLo_med[3 * o + c];
            if (S.unc_clamp[o]) {   /* the clamp taken the other way adds or removes this vertex's term */
                const double* Lc = tk < S.t_end[v] ? &S.Lo_med[3 * o] : &S.calt_Lo_med[3 * o];
                for (int c = 0; c < 3; ++c) bud[c] += w * ss * dt * T * fabs(Lc[c]);
            }
        }
        if (S.unc_prim[v]) {
            /* |L_i(alternative) - L_i(current)| of a near-tie primary ray */
            for (int c = 0; c < 3; ++c) {
                double cur = S.hit[v] >= 0 ? exp(-st * S.t_end[v]) * S.Lo_surf[3 * v + c] : 0.0;
                double alt = S.alt_hit[v] >= 0 ? exp(-st * S.alt_t[v]) * S.alt_Lo_surf[3 * v + c] : 0.0;
                for (int k = 1; k <= S.K; ++k) {
                    double tk = ((double)k - 0.5) * dt, T = exp(-st * tk);
                    size_t o = (size_t)(k - 1) * S.V + v;
                    if (tk < S.t_end[v]) cur += ss * dt * T * S.Lo_med[3 * o + c];
                    if (tk < S.alt_t[v]) alt += ss * dt * T * S.alt_Lo_med[3 * o + c];
                }
                bud[c] += w * fabs(alt - cur);
            }
        }
    }
    ffsum fs, fm;
    ff_accumulate(s, &S, p, x, 0, 0, &fs);
    ff_accumulate(s, &S, p, x, 1, S.K, &fm);
    double Ht[3][3][3];
    for (int c = 0; c < 3; ++c) {
        out[O_L + c] = Lss[c] + Lms[c];
        out[O_L_SS + c] = Lss[c];
        out[O_L_MS + c] = Lms[c];
        out[O_LFF + c] = fs.L[c] + fm.L[c];
        out[O_LFF_SS + c] = fs.L[c];
        out[O_LFF_MS + c] = fm.L[c];
        for (int i = 0; i < 3; ++i) {
            out[O_G + 3 * c + i] = fs.g[c][i] + fm.g[c][i];
            out[O_G_SS + 3 * c + i] = fs.g[c][i];
            out[O_G_MS + 3 * c + i] = fm.g[c][i];
            for (int j = 0; j < 3; ++j) Ht[c][i][j] = fs.H[c][i][j] + fm.H[c][i][j];
        }
        pack_h6(Ht[c], &out[O_H + 6 * c]);
        pack_h6(fs.H[c], &out[O_H_SS + 6 * c]);
        pack_h6(fm.H[c], &out[O_H_MS + 6 * c]);
        out[O_BUD_L + c] = bud[c];
        out[O_BUD_LFF + c] = fs.bud_L[c] + fm.bud_L[c];
        out[O_BUD_G + c] = fs.bud_g[c] + fm.bud_g[c];
        out[O_BUD_H + c] = fs.bud_H[c] + fm.bud_H[c];
    }
    /* radius from the luminance Hessian (Eq. radiusAniso3D, R15) */
    double HY[3][3], h6[6];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) HY[i][j] = LUM[0] * Ht[0][i][j] + LUM[1] * Ht[1][i][j] + LUM[2] * Ht[2][i][j];
    pack_h6(HY, h6);
    double LY = LUM[0] * out[O_L] + LUM[1] * out[O_L + 1] + LUM[2] * out[O_L + 2];
    int status = 0;
    double lam[3];
    out[O_R] = orc_radius(LY, h6, (double)p->eps, (double)p->r_min, (double)p->r_max, &status, lam);
    for (int i = 0; i < 3; ++i) out[O_EIG + i] = lam[i];
    double hn = 0.0;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) hn += HY[i][j] * HY[i][j];
    out[O_KAPPA] = (fs.sumHnorm + fm.sumHnorm) / sqrt(hn);
    for (int q = 0; q < O_BUD_L; ++q)
        if (q != O_KAPPA && q != O_MEDGE && q != O_MT && !isfinite(out[q])) status |= REC_NONFINITE;
    if (fs.n_degen + fm.n_degen) status |= REC_DEGENERATE;
    out[O_STATUS] = status;
    out[O_NSHELL] = S.K;
    double me = INFINITY, mt_ = INFINITY;
    int nprim = 0;
    for (int v = 0; v < S.V; ++v) {
        if (S.margin_e[v] < me) me = S.margin_e[v];
        if (S.tie[v] < mt_) mt_ = S.tie[v];
        nprim += S.unc_prim[v];
    }
    out[O_MEDGE] = me;
    out[O_MT] = mt_;
    out[O_NRAYS] = S.V;
    out[O_NDEGEN] = fs.n_degen + fm.n_degen;
    out[O_LY] = LY;
    out[O_LAMMAX] = fmax(fabs(lam[0]), fmax(fabs(lam[1]), fabs(lam[2])));
    out[O_N_PRIM_UNC] = nprim;
    out[O_N_UNC] = fs.n_unc + fm.n_unc;
    out[O_N_REPLAYED] = S.n_replayed;
    out[O_N_BAD_REPLAY] = S.n_bad_replay;
    out[O_N_LIT_REPLAYED] = S.n_lit_replayed;
    out[O_N_UNEXPLAINED] = S.n_unexplained;
    if (dbg_hit)
        for (int v = 0; v < S.V; ++v) {
            dbg_hit[v] = S.hit[v];
            dbg_t[v] = S.t_end[v];
            dbg_margin[v] = S.margin_e[v];
            dbg_tie[v] = S.tie[v];
        }
    if (dbg_lit) {      /* the visibility decisions: vertex v of shell k has radiance */
        int words = (dbg_stride + 31) / 32;
        for (int k = 0; k <= S.K && k < dbg_shells; ++k)
            for (int v = 0; v < S.V; ++v) {
                const double* Lo;
                double key;
                vertex_t(&S, p, k, v, &Lo, &key);
                if (Lo[0] != 0.0 || Lo[1] != 0.0 || Lo[2] != 0.0)
                    dbg_lit[(size_t)k * words + (v >> 5)] |= 1u << (v & 31);
            }
    }
    shells_free(&S);
}

/* ----------------------------------------------------------- thread pool */
typedef struct {
    const orc_scene* s;
    const orc_params* p;
    const float* pos;
    const int64_t* rec_ids;
    const int32_t* n_bands;
    int n;
    double* out;
    int32_t* dbg_hit;
    double *dbg_t, *dbg_margin, *dbg_tie;
    int dbg_stride;
    uint32_t* dbg_lit;
    int dbg_shells;
    orc_replay replay;
    volatile int next;
} job_t;

static void* worker(void* arg) {
    job_t* J = (job_t*)arg;
    for (;;) {
        int i = __sync_fetch_and_add(&J->next, 1);
        if (i >= J->n) break;
        int nb = J->n_bands ? J->n_bands[i] : J->p->n_bands;
        int ns = J->n_bands ? 2 * J->n_bands[i] : J->p->n_bins;
        int64_t rec = J->rec_ids ? J->rec_ids[i] : J->p->rec_base + i;
        size_t o = (size_t)i * J->dbg_stride;
        orc_replay R = J->replay;
        if (R.hit) R.hit += (size_t)i * R.stride;
        if (R.t) R.t += (size_t)i * R.stride;
        if (R.lit) R.lit += (size_t)i * R.shells * ((R.stride + 31) / 32);
        compute_record(J->s, J->p, ldv(J->pos + 3 * i), nb, ns, rec, R.hit ? &R : NULL,
                       J->out + (size_t)i * ORC_OUT_STRIDE,
                       J->dbg_hit ? J->dbg_hit + o : NULL, J->dbg_hit ? J->dbg_t + o : NULL,
                       J->dbg_hit ? J->dbg_margin + o : NULL, J->dbg_hit ? J->dbg_tie + o : NULL,
                       J->dbg_lit ? J->dbg_lit + (size_t)i * J->dbg_shells * ((J->dbg_stride + 31) / 32) : NULL,
                       J->dbg_shells, J->dbg_stride);
    }
    return NULL;
}

/* Compute n records.  rec_ids (nullable) gives each record's jitter index (default
 * rec_base + i); n_bands (nullable) gives per-record band counts with bins = 2 bands.
 * dbg_* (nullable) receive per-ray hit id, t_end, edge margin and tie gap, stride dbg_stride,
 * and the visibility bits (dbg_lit, zeroed by the caller, dbg_shells rows per record).
 * Replay (nullable pointers, see orc_replay): per record, replay_stride primary hit ids
 * (ray order, pole rays last, -1 = no hit), FP32 ray ends, and replay_shells rows of
 * (replay_stride + 31) / 32 visibility words. */
int orc_records(const orc_scene* s, const orc_params* p, const float* pos, const int64_t* rec_ids,
                const int32_t* n_bands, int n, double* out, int n_threads, int32_t* dbg_hit, double* dbg_t,
                double* dbg_margin, double* dbg_tie, int dbg_stride, uint32_t* dbg_lit, int dbg_shells,
                const int32_t* replay_hit, const float* replay_t, const uint32_t* replay_lit, int replay_stride,
                int replay_shells) {
    orc_replay R = {replay_hit, replay_t, replay_lit, replay_stride, replay_shells};
    job_t J = {s, p, pos, rec_ids, n_bands, n, out, dbg_hit, dbg_t, dbg_margin, dbg_tie, dbg_stride, dbg_lit,
               dbg_shells, R, 0};
    if (n_threads < 1) n_threads = 1;
    if (n_threads > 256) n_threads = 256;
    pthread_t th[256];
    for (int k = 0; k < n_threads; ++k) pthread_create(&th[k], NULL, worker, &J);
    for (int k = 0; k < n_threads; ++k) pthread_join(th[k], NULL);
    return 0;
}

/* Frozen-vertex evaluation (for finite-difference pins): the shells, vertex radiances
 * and furthest-vertex choices of the record at x0 are held fixed, and the triangulated
 * radiance L_ff and its analytic derivatives are evaluated at each x_eval.
 * out per point: L[3], grad[3][3], hess[3][3][3] (full) = 39 doubles. */
int orc_frozen_eval(const orc_scene* s, const orc_params* p, const float* x0f, int64_t rec, const double* x_eval,
                    int n_eval, int which, double* out) {
    shells_t S;
    build_shells(s, ldv(x0f), p, p->n_bands, p->n_bins, rec, NULL, &S);
    int k0 = which == 2 ? 1 : 0, k1 = which == 1 ? 0 : S.K;
    for (int e = 0; e < n_eval; ++e) {
        ffsum acc;
        ff_accumulate(s, &S, p, mk(x_eval[3 * e], x_eval[3 * e + 1], x_eval[3 * e + 2]), k0, k1, &acc);
        double* o = out + 39 * e;
        for (int c = 0; c < 3; ++c) {
            o[c] = acc.L[c];
            for (int i = 0; i < 3; ++i) o[3 + 3 * c + i] = acc.g[c][i];
            for (int i = 0; i < 3; ++i)
                for (int j = 0; j < 3; ++j) o[12 + 9 * c + 3 * i + j] = acc.H[c][i][j];
        }
    }
    int K = S.K;
    shells_free(&S);
    return K;
}

/* ------------------------------------------------- primitive exports for pins */
void orc_ray_directions(const orc_params* p, int64_t rec, double* out) {
    int V = p->n_bands * p->n_bins + 2;
    for (int v = 0; v < V; ++v) {
        v3 d = ray_direction(p, p->n_bands, p->n_bins, rec, v);
        out[3 * v] = d.x; out[3 * v + 1] = d.y; out[3 * v + 2] = d.z;
    }
}

double orc_jitter(uint64_t seed, int64_t rec, int i, int j, int stream) { return jitter(seed, rec, i, j, stream); }
uint64_t orc_splitmix64(uint64_t x) { return splitmix64(x); }

static void pack_sfun(const sfun* f, double* o) {
    o[0] = f->v;
    for (int i = 0; i < 3; ++i) o[1 + i] = f->g[i];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) o[4 + 3 * i + j] = f->H[i][j];
}

int orc_formfactor(const double* x, const double* y1, const double* y2, const double* y3, int ff_signed, double* out13) {
    sfun F;
    int ok = formfactor(mk(x[0], x[1], x[2]), mk(y1[0], y1[1], y1[2]), mk(y2[0], y2[1], y2[2]),
                        mk(y3[0], y3[1], y3[2]), ff_signed, &F);
    pack_sfun(&F, out13);
    return ok;
}

void orc_transmittance(const double* x, const double* y, double sigma_t, double* out13) {
    sfun T;
    transmittance(mk(x[0], x[1], x[2]), mk(y[0], y[1], y[2]), sigma_t, &T);
    pack_sfun(&T, out13);
}

void orc_phase(const double* x, const double* y, const double* wo, double g, double* out13) {
    sfun f;
    phase(mk(x[0], x[1], x[2]), mk(y[0], y[1], y[2]), mk(wo[0], wo[1], wo[2]), g, &f);
    pack_sfun(&f, out13);
}

/* out: L[3], grad[3][3], hess[3][3][3] (39 doubles); far_mask bit q marks vertex q as
 * one of the (tied) furthest vertices, Lo is [3][3] (radiance of each vertex) */
int orc_cell(const double* x, const double* y1, const double* y2, const double* y3, int far_mask, const double* Lo,
             double sigma_t, double g, const double* wo, double weight, int general, int ff_signed, double* out) {
    v3 y[3] = {mk(y1[0], y1[1], y1[2]), mk(y2[0], y2[1], y2[2]), mk(y3[0], y3[1], y3[2])};
    v3 yf[3];
    const double* Lf[3];
    int nf = 0;
    for (int q = 0; q < 3; ++q)
        if (far_mask & (1 << q)) { yf[nf] = y[q]; Lf[nf] = Lo + 3 * q; ++nf; }
    cellout co;
    int ok = cell_radiance(mk(x[0], x[1], x[2]), y[0], y[1], y[2], nf, yf, Lf, sigma_t, g, mk(wo[0], wo[1], wo[2]),
                           weight, general, ff_signed, &co, NULL, NULL);
    for (int c = 0; c < 3; ++c) {
        out[c] = co.L[c];
        for (int i = 0; i < 3; ++i) out[3 + 3 * c + i] = co.g[c][i];
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) out[12 + 9 * c + 3 * i + j] = co.H[c][i][j];
    }
    return ok;
}

/* closest hit of arbitrary rays (for traversal pins): id, t, margin, tie per ray */
void orc_trace(const orc_scene* s, const double* o, const double* d, int n, int32_t* id, double* t, double* margin,
               double* tie) {
    for (int i = 0; i < n; ++i) {
        double tt, mg = INFINITY, te = INFINITY, tv = INFINITY;
        id[i] = closest_hit(s, mk(o[3 * i], o[3 * i + 1], o[3 * i + 2]), mk(d[3 * i], d[3 * i + 1], d[3 * i + 2]),
                            &tt, &mg, &te, &tv, 1);
        t[i] = tt;
        margin[i] = mg;
        tie[i] = te;
    }
}

/* ------------------------------------------------ query (Eq. radianceTaylor) */
/* brute force over all records: C = {k : |x' - x_k| < R_k}, w = 3d^2 - 2d^3,
 * d = 1 - |x' - x_k| / R_k, out = sum w (L_k + grad L_k . D [+ D^T H_k D / 2]) / sum w.
 * status = |C| (0 = miss, out = 0).  near[q] = 1 when some |D| is within 1e-5 R of R. */
int orc_query(const double* rpos, const double* rR, const double* rL, const double* rgrad, const double* rhess,
              int n_rec, const double* q, int nq, int order, double* out, int32_t* status, int32_t* near) {
    for (int i = 0; i < nq; ++i) {
        v3 xq = mk(q[3 * i], q[3 * i + 1], q[3 * i + 2]);
        double acc[3] = {0, 0, 0}, sw = 0.0;
        int cnt = 0, nr = 0;
        for (int k = 0; k < n_rec; ++k) {
            v3 D = sub(xq, mk(rpos[3 * k], rpos[3 * k + 1], rpos[3 * k + 2]));
            double dist = norm(D), R = rR[k];
            if (fabs(dist - R) <= 1e-5 * R) nr = 1;
            if (!(dist < R)) continue;
            double dd = 1.0 - dist / R;
            double w = 3.0 * dd * dd - 2.0 * dd * dd * dd;
            for (int c = 0; c < 3; ++c) {
                const double* g = &rgrad[9 * k + 3 * c];
                double val = rL[3 * k + c] + g[0] * D.x + g[1] * D.y + g[2] * D.z;
                if (order == 2) {
                    const double* h = &rhess[18 * k + 6 * c];
                    double quad = h[0] * D.x * D.x + h[3] * D.y * D.y + h[5] * D.z * D.z +
                                  2.0 * (h[1] * D.x * D.y + h[2] * D.x * D.z + h[4] * D.y * D.z);
                    val += 0.5 * quad;
                }
                acc[c] += w * val;
            }
            sw += w;
            ++cnt;
        }
        for (int c = 0; c < 3; ++c) out[3 * i + c] = cnt ? acc[c] / sw : 0.0;
        status[i] = cnt;
        if (near) near[i] = nr;
    }
    return 0;
}

/* Eq. radianceTaylor over ellipsoidal records: the distance ratio |D|/R_k becomes the
 * ellipsoidal norm rho = sqrt(D^T M_k D) (M_k from orc_aniso), C = {k : rho < 1},
 * d = 1 - rho, w = 3d^2 - 2d^3; with M_k = I / R_k^2 this is orc_query.  near[q] = 1 when
 * some rho is within 1e-5 of 1.  metric [n_rec][6] upper triangles. */
int orc_query_aniso(const double* rpos, const double* metric, const double* rL, const double* rgrad,
                    const double* rhess, int n_rec, const double* q, int nq, int order, double* out,
                    int32_t* status, int32_t* near) {
    for (int i = 0; i < nq; ++i) {
        v3 xq = mk(q[3 * i], q[3 * i + 1], q[3 * i + 2]);
        double acc[3] = {0, 0, 0}, sw = 0.0;
        int cnt = 0, nr = 0;
        for (int k = 0; k < n_rec; ++k) {
            v3 D = sub(xq, mk(rpos[3 * k], rpos[3 * k + 1], rpos[3 * k + 2]));
            const double* m = &metric[6 * k];
            double r2 = m[0] * D.x * D.x + m[3] * D.y * D.y + m[5] * D.z * D.z +
                        2.0 * (m[1] * D.x * D.y + m[2] * D.x * D.z + m[4] * D.y * D.z);
            double rho = sqrt(fmax(r2, 0.0));
            if (fabs(rho - 1.0) <= 1e-5) nr = 1;
            if (!(rho < 1.0)) continue;
            double dd = 1.0 - rho;
            double w = 3.0 * dd * dd - 2.0 * dd * dd * dd;
            for (int c = 0; c < 3; ++c) {
                const double* g = &rgrad[9 * k + 3 * c];
                double val = rL[3 * k + c] + g[0] * D.x + g[1] * D.y + g[2] * D.z;
                if (order == 2) {
                    const double* h = &rhess[18 * k + 6 * c];
                    double quad = h[0] * D.x * D.x + h[3] * D.y * D.y + h[5] * D.z * D.z +
                                  2.0 * (h[1] * D.x * D.y + h[2] * D.x * D.z + h[4] * D.y * D.z);
                    val += 0.5 * quad;
                }
                acc[c] += w * val;
            }
            sw += w;
            ++cnt;
        }
        for (int c = 0; c < 3; ++c) out[3 * i + c] = cnt ? acc[c] / sw : 0.0;
        status[i] = cnt;
        if (near) near[i] = nr;
    }
    return 0;
}

int orc_out_stride(void) { return ORC_OUT_STRIDE; }

/* ------------------------------------------------ coarse features (learned radius) */
/* Not in the paper: the input of the learned radius predictor.  For the coarse ray set
 * (rays v < N of the n_bands x n_bins strata, jitter from p->seed): out[v] = log(t_end),
 * the distance to the first hit or to the cube exit; out[N + v] = sum over lights of
 * T(y, light) V(y, light) at y = x + t_end d (hit points start their shadow ray 1e-5 along
 * the normal facing x, exit points start at y).  unc[v] / unc[N + v] (nullable) flag
 * features whose ray or shadow ray is a near tie (within 1e-6 of an edge). */
int orc_coarse_features(const orc_scene* s, const orc_params* p, const float* pos, const int64_t* rec_ids, int n,
                        double* out, uint8_t* unc) {
    int nb = p->n_bands, ns = p->n_bins, N = nb * ns;
    for (int i = 0; i < n; ++i) {
        v3 x = ldv(pos + 3 * i);
        int64_t rec = rec_ids ? rec_ids[i] : p->rec_base + i;
        for (int v = 0; v < N; ++v) {
            v3 d = ray_direction(p, nb, ns, rec, v);
            double t, mg = INFINITY, tie = INFINITY, tv = INFINITY;
            int id = closest_hit(s, x, d, &t, &mg, &tie, &tv, 1);
            int u_prim = mg < TIE_EDGE || tv < TIE_T;
            if (id < 0) t = cube_exit(x, d);
            v3 y = add(x, scl(d, t));
            v3 o = y;
            if (id >= 0) {
                v3 a = ldv(s->in.tri_v + 9 * id), b = ldv(s->in.tri_v + 9 * id + 3), c = ldv(s->in.tri_v + 9 * id + 6);
                v3 nn = cross(sub(b, a), sub(c, a));
                nn = scl(nn, 1.0 / norm(nn));
                if (dot(nn, d) > 0) nn = scl(nn, -1.0);
                o = add(y, scl(nn, ORC_SHADOW_OFFSET));
            }
            double tv_sum = 0.0, margin = INFINITY;
            for (int L = 0; L < s->in.n_lights; ++L) {
                v3 pl = ldv(s->in.light_pos + 3 * L);
                v3 lo = sub(pl, o);
                double dl = norm(lo);
                if (!occluded(s, o, scl(lo, 1.0 / dl), dl, &margin, 1)) tv_sum += exp(-s->sigma_t * norm(sub(pl, y)));
            }
            out[(size_t)i * 2 * N + v] = log(t);
            out[(size_t)i * 2 * N + N + v] = tv_sum;
            if (unc) {
                unc[(size_t)i * 2 * N + v] = (uint8_t)u_prim;
                unc[(size_t)i * 2 * N + N + v] = (uint8_t)(u_prim || margin < TIE_EDGE);
            }
        }
    }
    return 0;
}
