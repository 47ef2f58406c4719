// vrc_internal.cuh -- device data layout and device helpers shared by the library's
// kernels: the scene in HBM, the counter-based jitter, the stratified ray
// directions, and bounding-volume-hierarchy ray casting.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "vrc.h"

#define VRC_PI_F 3.14159265358979323846f

// ------------------------------------------------------------------ scene in HBM
// BVH node: 64 bytes, both children's boxes side by side so one node fetch tests
// two boxes:  n0 = (c0.lo.x, c0.hi.x, c0.lo.y, c0.hi.y)
//             n1 = (c1.lo.x, c1.hi.x, c1.lo.y, c1.hi.y)
//             n2 = (c0.lo.z, c0.hi.z, c1.lo.z, c1.hi.z)
//             n3 = (child0, child1, -, -) as int bits.
// child >= 0: inner node index; child < 0: leaf, -(1 + (first << 3 | (count - 1))).
// Triangles (BVH leaf order): 3 float4 = (v0, prim id bits), (e1 = v1 - v0, 0), (e2 = v2 - v0, 0).
// Per original primitive: 3 float4 = (unit normal, 0), (albedo rgb, 0), (emission rgb, 0).
// Light buffer (one per point light): a cube map of directions around the light,
// R x R cells per face; cell c lists (triangle index in BVH order, lower bound of the
// triangle's distance to the light) for every triangle whose projection from the light
// overlaps the cell, sorted by that distance.  A shadow segment from y to the light can
// only meet triangles listed in the cell of direction y - light that are nearer than y.
struct DevLightBuf {
    // per cell: first and one-past-last entry, then float bits of (a) the first entry's
    // distance bound (+inf for an empty cell) and (b) a distance beyond which every point
    // of the cell is behind one triangle that covers the whole cell (+inf if none does)
    const int4* __restrict__ cell;      // [6 R R]
    const int2* __restrict__ ent;       // (tri, float bits of the distance bound)
    int R;
};

struct DevScene {
    const float4* __restrict__ nodes;
    const float4* __restrict__ tris;
    const float4* __restrict__ prim;
    int n_nodes, n_tris, n_lights;
    float3 lpos[VRC_MAX_LIGHTS];
    float3 lI[VRC_MAX_LIGHTS];
    DevLightBuf lb[VRC_MAX_LIGHTS];
    int use_lb;                         // 1: shadow rays use the light buffers
    float sigma_s, sigma_t, g;
};

struct vrc_scene {
    DevScene dev;
    float4* d_nodes;
    float4* d_tris;
    float4* d_prim;
    int4* d_lb_cell[VRC_MAX_LIGHTS];
    int2* d_lb_ent[VRC_MAX_LIGHTS];
    long long lb_entries;
    int n_prims;
    vrc_record_tuning tuning;
    int sm_count;
    int* d_counter;       // persistent-launch work counter (one int)
    int* d_order;         // largest-first record order + histogram (grown on demand)
    int order_cap;
    // per-kernel timing of record launches (vrc_record_kernel_times): event triples, one
    // per launch since the last read; recorded only while enabled and not capturing
    int timing;
    int n_timed;
    cudaEvent_t t_ev[64][4];
    int t_ev_made;
    float4* d_pre_ray;    // primary pre-pass: (direction, t_end) per ray (grown on demand)
    float* d_pre_Lo;      // primary pre-pass: surface radiance rgb per ray
    long long pre_cap;    // rays the pre-pass buffers hold
    // device staging for vrc_compute_records_host (grown on demand)
    float* h_stage_dev;
    size_t h_stage_floats;
    // vrc_cache_step_host: query staging (grown on demand), a side stream for the copies
    // that overlap the kernels, and the two events that order it against the main stream
    float* q_stage_dev;
    size_t q_stage_floats;
    cudaStream_t step_st[2];
    cudaEvent_t step_ev[2];
    int step_made;
};

// Record grid (query.cu builds it; the renderer reads it): compact record rows and a
// uniform grid over the unit cube with CSR lists of the records overlapping each cell.
struct vrc_grid {
    int n;                 // records
    int G;                 // cells per axis
    int order;             // 1 or 2
    float4* rec;           // [n][4]: (pos, R), (L, g_r.x), (g_r.y, g_r.z, g_g.x, g_g.y), (g_g.z, g_b)
    float4* hess;          // [n][5]: 18 Hessian entries (order 2), padded
    int aniso;             // 1: ellipsoidal records (rec .w = largest principal radius)
    float4* ell;           // [n][2]: region matrix M (xx, xy, xz, yy), (yz, zz, -, -) when aniso
    float4* ext;           // [n]: bounding-box half extents and largest radius when aniso
    int* cell_start;       // [G^3 + 1]
    int* cell_list;        // [entries]
    long long entries;
    // query scratch (grown on demand)
    int* q_cell;           // [cap]
    int* q_rank;           // [cap]
    float4* q_pts;         // [cap] the query points in cell order, .w = the query's index
    int* q_count;          // [G^3 + 1]
    int* scan_tmp;         // block sums
    int q_cap;
    // capacities of the buffers above (elements), kept across vrc_rebuild_record_grid
    long long rec_cap, hess_cap, ell_cap, cell_cap, scan_cap, list_cap, q_count_cap;
};

// ------------------------------------------------------------------ small vector ops
__device__ __forceinline__ float3 f3(float x, float y, float z) { return make_float3(x, y, z); }
__device__ __forceinline__ float3 operator+(float3 a, float3 b) { return f3(a.x + b.x, a.y + b.y, a.z + b.z); }
__device__ __forceinline__ float3 operator-(float3 a, float3 b) { return f3(a.x - b.x, a.y - b.y, a.z - b.z); }
__device__ __forceinline__ float3 operator*(float3 a, float s) { return f3(a.x * s, a.y * s, a.z * s); }
__device__ __forceinline__ float dot3(float3 a, float3 b) { return fmaf(a.x, b.x, fmaf(a.y, b.y, a.z * b.z)); }
__device__ __forceinline__ float3 cross3(float3 a, float3 b) {
    return f3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}

// ------------------------------------------------------------------ jitter
// splitmix64 (Steele, Lea, Flood 2014; Vigna's finaliser constants) on a counter key
// built from the seed, record, band, bin and stream; the top 24 bits give u in [0,1)
// exactly representable in float.
__device__ __forceinline__ uint64_t splitmix64_dev(uint64_t x) {
    uint64_t z = x + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
__device__ __forceinline__ float jitter_dev(uint64_t seed, int64_t rec, int i, int j, int stream) {
    uint64_t key = seed ^ ((uint64_t)rec << 32) ^ ((uint64_t)i << 16) ^ (uint64_t)j ^ ((uint64_t)stream << 60);
    return (float)(uint32_t)(splitmix64_dev(key) >> 40) * (1.0f / 16777216.0f);
}

// ------------------------------------------------------------------ stratified ray set
// Direction of stratum (band i, bin j): cos(theta) = 1 - 2 (i + u1) / nb, phi = 2 pi (j + u2) / ns.
// Written so the float result stays within ~1e-7 of the exact direction: 1 - cos and
// 1 + cos are formed from integer-exact pieces (no rounding of i + u1), and phi is the
// bin start (quadrant-reduced, exact integer arithmetic) rotated by the in-bin offset.
__device__ __forceinline__ float3 stratum_direction(int i, int j, int nb, int ns, float u1, float u2) {
    float inb = 1.0f / (float)nb;
    float ct, st;
    if (2 * i < nb) {
        float w = fmaf(2.0f * u1, inb, (float)(2 * i) * inb);          // 1 - cos, in [0, 1]
        ct = 1.0f - w;
        st = sqrtf(fmaxf(0.0f, w * (2.0f - w)));
    } else {
        float v = fmaf(-2.0f * u1, inb, (float)(2 * (nb - i)) * inb);  // 1 + cos
        ct = v - 1.0f;
        st = sqrtf(fmaxf(0.0f, v * (2.0f - v)));
    }
    int q4 = 4 * j;
    int quad = q4 / ns;                 // bin start angle = (pi/2) (quad + rem/ns)
    int rem = q4 - quad * ns;
    float s0, c0;
    sincospif(0.5f * (float)rem / (float)ns, &s0, &c0);
    float cq, sq;
    switch (quad & 3) {
        case 0: cq = c0; sq = s0; break;
        case 1: cq = -s0; sq = c0; break;
        case 2: cq = -c0; sq = -s0; break;
        default: cq = s0; sq = -c0; break;
    }
    float sd, cd;
    sincospif(2.0f * u2 / (float)ns, &sd, &cd);   // in-bin offset 2 pi u2 / ns
    float cp = cq * cd - sq * sd;
    float sp = sq * cd + cq * sd;
    return f3(st * cp, st * sp, ct);
}

__device__ __forceinline__ float3 ray_direction_dev(uint64_t seed, int64_t rec, int v, int nb, int ns) {
    int n = nb * ns;
    if (v == n) return f3(0.f, 0.f, 1.f);
    if (v == n + 1) return f3(0.f, 0.f, -1.f);
    int i = v / ns, j = v - (v / ns) * ns;
    return stratum_direction(i, j, nb, ns, jitter_dev(seed, rec, i, j, 0), jitter_dev(seed, rec, i, j, 1));
}

// distance to leave the unit cube from inside
__device__ __forceinline__ float cube_exit_dev(float3 o, float3 d) {
    float t = 3.0e38f;
    if (d.x > 0.f) t = fminf(t, (1.f - o.x) / d.x); else if (d.x < 0.f) t = fminf(t, -o.x / d.x);
    if (d.y > 0.f) t = fminf(t, (1.f - o.y) / d.y); else if (d.y < 0.f) t = fminf(t, -o.y / d.y);
    if (d.z > 0.f) t = fminf(t, (1.f - o.z) / d.z); else if (d.z < 0.f) t = fminf(t, -o.z / d.z);
    return t;
}

// ------------------------------------------------------------------ ray casting
#define VRC_TMIN 1e-6f
#define VRC_BARY_EPS 2e-7f      // closes float cracks between triangles sharing an edge
#define VRC_STACK 64

// Moller-Trumbore against one triangle; barycentrics widened by VRC_BARY_EPS.
__device__ __forceinline__ bool tri_hit(const float4* __restrict__ T, int k, float3 o, float3 d, float tmin,
                                        float tmax, float* t_out, int* id_out) {
    float4 a = __ldg(&T[3 * k]), b = __ldg(&T[3 * k + 1]), c = __ldg(&T[3 * k + 2]);
    float3 v0 = f3(a.x, a.y, a.z), e1 = f3(b.x, b.y, b.z), e2 = f3(c.x, c.y, c.z);
    float3 p = cross3(d, e2);
    float det = dot3(e1, p);
    if (det == 0.f) return false;
    float inv = 1.0f / det;
    float3 s = o - v0;
    float u = dot3(s, p) * inv;
    if (u < -VRC_BARY_EPS || u > 1.f + VRC_BARY_EPS) return false;
    float3 q = cross3(s, e1);
    float v = dot3(d, q) * inv;
    if (v < -VRC_BARY_EPS || u + v > 1.f + VRC_BARY_EPS) return false;
    float t = dot3(e2, q) * inv;
    if (!(t > tmin && t < tmax)) return false;
    *t_out = t;
    *id_out = __float_as_int(a.w);
    return true;
}

// Closest hit (ANY = false) or any hit (ANY = true) along o + t d, t in (tmin, tmax).
// Closest-hit ties go to the lowest primitive id.  Returns the primitive id or -1;
// t_hit receives the hit parameter.  Stack-based traversal of the two-wide BVH,
// nearer child first.
template <bool ANY>
__device__ int bvh_trace(const DevScene& sc, float3 o, float3 d, float tmin, float tmax, float* t_hit) {
    if (sc.n_tris == 0) return -1;
    const float big = 1e30f;
    float3 inv = f3(fabsf(d.x) > 1e-30f ? 1.0f / d.x : copysignf(big, d.x),
                    fabsf(d.y) > 1e-30f ? 1.0f / d.y : copysignf(big, d.y),
                    fabsf(d.z) > 1e-30f ? 1.0f / d.z : copysignf(big, d.z));
    float3 oi = f3(o.x * inv.x, o.y * inv.y, o.z * inv.z);
    int best = -1;
    float best_t = tmax;
    int stack[VRC_STACK];
    int sp = 0;
    int code = 0;
    while (true) {
        if (code >= 0) {
            const float4* N = sc.nodes + 4 * code;
            float4 n0 = __ldg(N), n1 = __ldg(N + 1), n2 = __ldg(N + 2), n3 = __ldg(N + 3);
            float a0 = fmaf(n0.x, inv.x, -oi.x), a1 = fmaf(n0.y, inv.x, -oi.x);
            float b0 = fmaf(n0.z, inv.y, -oi.y), b1 = fmaf(n0.w, inv.y, -oi.y);
            float z0 = fmaf(n2.x, inv.z, -oi.z), z1 = fmaf(n2.y, inv.z, -oi.z);
            float tn0 = fmaxf(fmaxf(fminf(a0, a1), fminf(b0, b1)), fmaxf(fminf(z0, z1), tmin));
            float tf0 = fminf(fminf(fmaxf(a0, a1), fmaxf(b0, b1)), fminf(fmaxf(z0, z1), best_t));
            a0 = fmaf(n1.x, inv.x, -oi.x); a1 = fmaf(n1.y, inv.x, -oi.x);
            b0 = fmaf(n1.z, inv.y, -oi.y); b1 = fmaf(n1.w, inv.y, -oi.y);
            z0 = fmaf(n2.z, inv.z, -oi.z); z1 = fmaf(n2.w, inv.z, -oi.z);
            float tn1 = fmaxf(fmaxf(fminf(a0, a1), fminf(b0, b1)), fmaxf(fminf(z0, z1), tmin));
            float tf1 = fminf(fminf(fmaxf(a0, a1), fmaxf(b0, b1)), fminf(fmaxf(z0, z1), best_t));
            bool h0 = tn0 <= tf0, h1 = tn1 <= tf1;
            int c0 = __float_as_int(n3.x), c1 = __float_as_int(n3.y);
            if (h0 && h1) {
                int nearc = tn0 <= tn1 ? c0 : c1, farc = tn0 <= tn1 ? c1 : c0;
                if (sp < VRC_STACK) stack[sp++] = farc;
                code = nearc;
            } else if (h0) {
                code = c0;
            } else if (h1) {
                code = c1;
            } else {
                if (sp == 0) break;
                code = stack[--sp];
            }
        } else {
            int z = -code - 1;
            int first = z >> 3, count = (z & 7) + 1;
            for (int k = first; k < first + count; ++k) {
                float t;
                int id;
                if (tri_hit(sc.tris, k, o, d, tmin, ANY ? tmax : best_t * (1.0f + 1e-7f) + 1e-30f, &t, &id)) {
                    if (ANY) {
                        *t_hit = t;
                        return id;
                    }
                    if (t < best_t || (t == best_t && id < best)) {
                        best_t = t;
                        best = id;
                    }
                }
            }
            if (sp == 0) break;
            code = stack[--sp];
        }
    }
    *t_hit = best_t;
    return best;
}

// cube-map cell of direction w (from the light): major axis (ties: x, then y), face =
// 2 axis + (negative ? 1 : 0), then the two other coordinates over |major| in [-1, 1]
__device__ __forceinline__ int lightbuf_cell(float3 w, int R) {
    float ax = fabsf(w.x), ay = fabsf(w.y), az = fabsf(w.z);
    int axis;
    float m, a, b, s;
    if (ax >= ay && ax >= az) { axis = 0; m = ax; s = w.x; a = w.y; b = w.z; }
    else if (ay >= az) { axis = 1; m = ay; s = w.y; a = w.z; b = w.x; }
    else { axis = 2; m = az; s = w.z; a = w.x; b = w.y; }
    int face = 2 * axis + (s < 0.f ? 1 : 0);
    float im = 1.0f / m;
    int i = min(R - 1, max(0, (int)floorf((a * im + 1.0f) * 0.5f * R)));
    int j = min(R - 1, max(0, (int)floorf((b * im + 1.0f) * 0.5f * R)));
    return (face * R + i) * R + j;
}

// Any hit on the segment from o toward light l (unit direction ld, length dist): the same
// triangle test as bvh_trace<true>, over the light-buffer candidates nearer than o.  Two
// per-cell bounds settle most points with one load and give the loop's own answer: a point
// no further than the first candidate's bound is lit (the loop would stop there), and a
// point beyond the covered distance is behind a triangle that every direction of the cell
// crosses well inside its edges (the loop would find it, or an earlier hit).
__device__ __forceinline__ bool lightbuf_occluded(const DevScene& sc, int l, float3 o, float3 ld, float dist) {
    const DevLightBuf& L = sc.lb[l];
    float3 w = o - sc.lpos[l];
    int c = lightbuf_cell(w, L.R);
    const int4 cd = __ldg(&L.cell[c]);
    if (!(dist > __int_as_float(cd.z))) return false;
    if (dist > __int_as_float(cd.w)) return true;
    for (int p = cd.x; p < cd.y; ++p) {
        int2 en = __ldg(&L.ent[p]);
        if (__int_as_float(en.y) >= dist) break;
        float t;
        int id;
        if (tri_hit(sc.tris, en.x, o, ld, VRC_TMIN, dist, &t, &id)) return true;
    }
    return false;
}

__device__ __forceinline__ bool shadow_occluded(const DevScene& sc, int l, float3 o, float3 ld, float dist) {
    if (sc.use_lb) return lightbuf_occluded(sc, l, o, ld, dist);
    float th;
    return bvh_trace<true>(sc, o, ld, VRC_TMIN, dist, &th) >= 0;
}

// ------------------------------------------------------------------ Henyey-Greenstein
__device__ __forceinline__ float hg_dev(float mu, float g) {
    float q = fmaf(-2.0f * g, mu, fmaf(g, g, 1.0f));
    float rq = rsqrtf(q);
    return (1.0f - g * g) * (0.25f / VRC_PI_F) * rq * rq * rq;
}

#define VRC_CUDA_CHECK(call)                           \
    do {                                               \
        cudaError_t e_ = (call);                       \
        if (e_ != cudaSuccess) return VRC_ERR_CUDA;    \
    } while (0)
