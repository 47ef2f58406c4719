// records.cu -- cache records: in-scattered radiance, occlusion-aware gradient and
// Hessian, and validity radius (Secs. 4-5, App. A and App. C of Marco et al. 2018).
//
// One thread block computes one record at a time (persistent blocks pull record ids
// from a work counter).  The record's stratified ray set is processed in chunks of
// bands so that the vertex ring of a chunk fits in shared memory:
//   1. primary phase   trace every ray of the chunk (closest hit); surface radiance at
//                      each hit with a shadow ray per light; Monte Carlo surface term.
//   2. surface shell   every cell of the chunk's triangulation at the hit points.
//   3. medium shells   for t_k = (k - 1/2) dt: vertex phase (a shadow ray from every
//                      unclamped vertex; vertices beyond their hit sit on the hit with
//                      zero radiance), Monte Carlo medium term, then the cell phase.
// Each cell yields 32 numbers (L, grad L, H L for 3 channels, the luminance-Hessian
// norm and a degeneracy flag) in FP32; a warp-transposed butterfly reduces 32 cells
// so that lane l owns the sum of value l, which it adds to a Neumaier-compensated
// accumulator (surface shell and medium shells kept apart).  The block's 32 sums are
// combined at the end; one thread then solves the 3x3 luminance-Hessian eigenproblem
// in FP64 and sets the radius.
#include <cmath>
#include <cstdio>
#include <mutex>
#include <vector>

#include "vrc_internal.cuh"

namespace {

struct RecArgs {
    const float* pos;
    int n;
    const int* n_bands;          // nullable: per-record bands, bins = 2 * bands
    int nb0, ns0;                // uniform bands / bins
    float dt, eps;
    float3 wo;
    uint64_t seed;
    int ff_signed;
    float r_min, r_max;
    long long rec_base;
    vrc_records_view out;
    int chunk_bands;             // bands per chunk
    int cap;                     // shared-memory vertex capacity per chunk
    int* counter;                // work counter (reset before the launch)
    const int* order;            // nullable: work item -> record (largest ray sets first)
    int parts;                   // 0 all shells, 1 surface shell only, 2 medium shells only
    const float4* pre_ray;       // nullable: primary pre-pass results of the current batch,
                                 // [item - item_base][pre_stride]
    const float* pre_Lo;         // [item - item_base][pre_stride][3]
    int pre_stride;              // rays per pre-pass slot (the largest ray set of the launch)
    int item_base, item_end;     // work items of the current batch (positions in `order`)
    int lo_grad;                 // medium vertices' radiance varies with x (one light)
};

__device__ __forceinline__ void neumaier(float& s, float& c, float x) {
    float t = s + x;
    if (fabsf(s) >= fabsf(x)) c += (s - t) + x;
    else c += (x - t) + s;
    s = t;
}

// lane l of the warp receives the sum over the warp of v[l] (v is 32 values per lane)
__device__ __forceinline__ float warp_transpose_reduce(float (&v)[32], int lane) {
#pragma unroll
    for (int s = 16; s >= 1; s >>= 1) {
        bool up = (lane & s) != 0;
#pragma unroll
        for (int i = 0; i < s; ++i) {
            float send = up ? v[i] : v[i + s];
            float keep = up ? v[i + s] : v[i];
            v[i] = keep + __shfl_xor_sync(0xffffffffu, send, s);
        }
    }
    return v[0];
}

// ----------------------------------------------------------------- vertex radiance
// Medium vertex: single scattering from the point lights (bounce limit, Sec. 6).
__device__ float3 medium_radiance(const DevScene& sc, float3 y, float3 d) {
    float3 L = f3(0.f, 0.f, 0.f);
    for (int l = 0; l < sc.n_lights; ++l) {
        float3 lv = sc.lpos[l] - y;
        float d2 = dot3(lv, lv);
        float dist = sqrtf(d2);
        float3 lh = lv * (1.0f / dist);
        if (shadow_occluded(sc, l, y, lh, dist)) continue;
        float f = hg_dev(dot3(lh, d), sc.g);      // light p_L -> y, then y -> x along -d
        float w = f * __expf(-sc.sigma_t * dist) / d2;
        L = L + sc.lI[l] * w;
    }
    return L;
}

// Surface vertex: Lambertian, two-sided (the light must be on the record's side),
// plus emission.
__device__ float3 surface_radiance(const DevScene& sc, int prim, float3 y, float3 d) {
    float4 n4 = __ldg(&sc.prim[3 * prim]);
    float4 al = __ldg(&sc.prim[3 * prim + 1]);
    float4 em = __ldg(&sc.prim[3 * prim + 2]);
    float3 n = f3(n4.x, n4.y, n4.z);
    if (dot3(n, d) > 0.f) n = n * -1.0f;
    float3 L = f3(em.x, em.y, em.z);
    for (int l = 0; l < sc.n_lights; ++l) {
        float3 lv = sc.lpos[l] - y;
        float d2 = dot3(lv, lv);
        float dist = sqrtf(d2);
        float cs = dot3(n, lv) / dist;
        if (cs <= 0.f) continue;
        float3 o = y + n * 1e-5f;
        float3 lo = sc.lpos[l] - o;
        float dl = sqrtf(dot3(lo, lo));
        if (shadow_occluded(sc, l, o, lo * (1.0f / dl), dl)) continue;
        float w = cs * __expf(-sc.sigma_t * dist) / (d2 * VRC_PI_F);
        L = L + f3(al.x * sc.lI[l].x, al.y * sc.lI[l].y, al.z * sc.lI[l].z) * w;
    }
    return L;
}

// HG phase f(w_i . wo) with w_i = w / |w|, w = x - y (a point y seen from x), and its
// gradient and Hessian (6 entries) with respect to x
__device__ __forceinline__ void hg_dx(float3 w, float3 wo, float g, float& fv, float (&gf)[3], float (&Hf)[6]) {
    float iw = rsqrtf(dot3(w, w));
    float3 wi = w * iw;
    float mu = dot3(wi, wo);
    float q = fmaf(-2.0f * g, mu, fmaf(g, g, 1.0f));
    float rq = rsqrtf(q);
    float cg = (1.0f - g * g) * (0.25f / VRC_PI_F);
    float rq3 = rq * rq * rq;
    fv = cg * rq3;
    float f1 = 3.0f * g * cg * rq3 * rq * rq;             // df/dmu
    float f2 = 5.0f * g * f1 * rq * rq;                   // d2f/dmu2
    float3 gm = (wo - wi * mu) * iw;                      // grad mu
    float iw2 = iw * iw;
    // H mu = (-wo wi^T - wi wo^T - mu I + 3 mu wi wi^T) / |w|^2
    float Hm[6] = {(-2.f * wo.x * wi.x - mu + 3.f * mu * wi.x * wi.x) * iw2,
                   (-wo.x * wi.y - wi.x * wo.y + 3.f * mu * wi.x * wi.y) * iw2,
                   (-wo.x * wi.z - wi.x * wo.z + 3.f * mu * wi.x * wi.z) * iw2,
                   (-2.f * wo.y * wi.y - mu + 3.f * mu * wi.y * wi.y) * iw2,
                   (-wo.y * wi.z - wi.y * wo.z + 3.f * mu * wi.y * wi.z) * iw2,
                   (-2.f * wo.z * wi.z - mu + 3.f * mu * wi.z * wi.z) * iw2};
    gf[0] = f1 * gm.x; gf[1] = f1 * gm.y; gf[2] = f1 * gm.z;
    Hf[0] = f2 * gm.x * gm.x + f1 * Hm[0];
    Hf[1] = f2 * gm.x * gm.y + f1 * Hm[1];
    Hf[2] = f2 * gm.x * gm.z + f1 * Hm[2];
    Hf[3] = f2 * gm.y * gm.y + f1 * Hm[3];
    Hf[4] = f2 * gm.y * gm.z + f1 * Hm[4];
    Hf[5] = f2 * gm.z * gm.z + f1 * Hm[5];
}

// ----------------------------------------------------------------- one cell
// Cell j with vertices r_q = y_q - x (q = 0..2) at ray parameters t_q and radiance
// Lo_q.  Writes the 32 values: L_j (3), grad L_j (3 x 3), H L_j (3 x 6), the Frobenius
// norm of the luminance Hessian, and 1 in v[31] for a degenerate cell (A = B = 0).
// Returns the number of tied furthest vertices evaluated (0: dark or degenerate cell).
//   L_j = f(w_c) Omega_j (1/m) sum_{q tied furthest} Lo_q T(|r_q|)
// Omega = 2 atan2(A, B) (Van Oosterom-Strackee) with A = r1 . (r2 x r3),
// B = r1 r2 r3 + (r1.r2) r3 + (r2.r3) r1 + (r1.r3) r2, grad A = -(r2-r1) x (r3-r1),
// H A = 0.  Here grad B = -sum_i c_i r_i with c_i = (rho_j rho_k + r_j.r_k)/rho_i + rho_j
// + rho_k, and H B = (sum c_i) I - sum_i r_i grad c_i^T; the Hessian of Omega is the
// symmetric form 2[-A HB/D - (2/D^2)(AB(aa^T - bb^T) + (B^2-A^2)/2 (ab^T + ba^T))].
// LOG (lo_grad, medium shells): a furthest vertex's radiance toward x is L_o(x_c) u(x), u the
// HG phase of its light toward x over its value toward the centre (u = 1 at x); u folds into
// the transmittance factor by the product rule (Eq. reducedRadianceDerivatives with grad L_o
// kept), for the open vertices (medium points: bit q of open_mask; a clamped vertex is a
// Lambertian surface point, constant toward x).  xl = x - (the light's position).
template <bool LOG>
__device__ __forceinline__ int cell_eval(const float3 (&r)[3], const float (&t)[3], const float3 (&Lo)[3],
                                         float sigma_t, float g, float3 wo, int ff_signed, float (&v)[32],
                                         float3 xl = f3(0.f, 0.f, 0.f), unsigned open_mask = 0u) {
    float tmx = fmaxf(t[0], fmaxf(t[1], t[2]));
    bool far0 = t[0] == tmx, far1 = t[1] == tmx, far2 = t[2] == tmx;
    bool lit = (far0 && (Lo[0].x != 0.f || Lo[0].y != 0.f || Lo[0].z != 0.f)) ||
               (far1 && (Lo[1].x != 0.f || Lo[1].y != 0.f || Lo[1].z != 0.f)) ||
               (far2 && (Lo[2].x != 0.f || Lo[2].y != 0.f || Lo[2].z != 0.f));
    if (!lit) return 0;
    // ---- solid angle and its derivatives
    float rho[3];
#pragma unroll
    for (int q = 0; q < 3; ++q) rho[q] = sqrtf(dot3(r[q], r[q]));
    // The plane normal (the same vector from any vertex, cyclic order kept) is taken from
    // the vertex nearest to x: from a far vertex of a sliver cell across a depth
    // discontinuity the two edges are long and nearly parallel, and their cross product
    // cancels in FP32 (a few percent of such a cell's Hessian near a surface).
    const bool b0 = rho[0] <= rho[1] && rho[0] <= rho[2];
    const bool b1 = !b0 && rho[1] <= rho[2];
    const float3 rb = b0 ? r[0] : (b1 ? r[1] : r[2]);
    const float3 rn = b0 ? r[1] : (b1 ? r[2] : r[0]);
    const float3 rp = b0 ? r[2] : (b1 ? r[0] : r[1]);
    float3 nrm = cross3(rn - rb, rp - rb);
    float A = dot3(rb, nrm);
    float3 a = nrm * -1.0f;
    if (!ff_signed && A < 0.f) { A = -A; a = nrm; }
    float d01 = dot3(r[0], r[1]), d12 = dot3(r[1], r[2]), d02 = dot3(r[0], r[2]);
    float B = fmaf(rho[0] * rho[1], rho[2], fmaf(d01, rho[2], fmaf(d12, rho[0], d02 * rho[1])));
    float D = fmaf(A, A, B * B);
    if (!(D > 1e-36f)) { v[31] = 1.0f; return 0; }
    float c[3];
    float3 gc[3];
    float dd[3] = {d12, d02, d01};   // r_j . r_k for the other two of i
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        int j = (i + 1) % 3, k = (i + 2) % 3;
        float ir = 1.0f / rho[i];
        float P = fmaf(rho[j], rho[k], dd[i]);
        c[i] = fmaf(P, ir, rho[j] + rho[k]);
        float irj = 1.0f / rho[j], irk = 1.0f / rho[k];
        // grad c_i = (-rho_k u_j - rho_j u_k - r_j - r_k)/rho_i + P u_i/rho_i^2 - u_j - u_k
        float aj = -(rho[k] * irj + 1.0f) * ir - irj;   // coefficient of r_j
        float ak = -(rho[j] * irk + 1.0f) * ir - irk;   // coefficient of r_k
        float ai = P * ir * ir * ir;                    // coefficient of r_i
        gc[i] = r[j] * aj + r[k] * ak + r[i] * ai;
    }
    float3 b = (r[0] * c[0] + r[1] * c[1] + r[2] * c[2]) * -1.0f;
    float csum = c[0] + c[1] + c[2];
    // H B, 6 unique entries (xx, xy, xz, yy, yz, zz)
    float HB[6];
    HB[0] = csum - (r[0].x * gc[0].x + r[1].x * gc[1].x + r[2].x * gc[2].x);
    HB[1] = -(r[0].x * gc[0].y + r[1].x * gc[1].y + r[2].x * gc[2].y);
    HB[2] = -(r[0].x * gc[0].z + r[1].x * gc[1].z + r[2].x * gc[2].z);
    HB[3] = csum - (r[0].y * gc[0].y + r[1].y * gc[1].y + r[2].y * gc[2].y);
    HB[4] = -(r[0].y * gc[0].z + r[1].y * gc[1].z + r[2].y * gc[2].z);
    HB[5] = csum - (r[0].z * gc[0].z + r[1].z * gc[1].z + r[2].z * gc[2].z);
    float iD = 1.0f / D;
    float Om = 2.0f * atan2f(A, B);
    float3 gO = (a * B - b * A) * (2.0f * iD);
    float k1 = -2.0f * A * iD;                       // coefficient of H B
    float k2 = -4.0f * iD * iD * A * B;              // of (aa^T - bb^T)
    float k3 = -2.0f * iD * iD * (B * B - A * A);    // of (ab^T + ba^T)
    float HO[6];
    HO[0] = k1 * HB[0] + k2 * (a.x * a.x - b.x * b.x) + k3 * 2.0f * a.x * b.x;
    HO[1] = k1 * HB[1] + k2 * (a.x * a.y - b.x * b.y) + k3 * (a.x * b.y + b.x * a.y);
    HO[2] = k1 * HB[2] + k2 * (a.x * a.z - b.x * b.z) + k3 * (a.x * b.z + b.x * a.z);
    HO[3] = k1 * HB[3] + k2 * (a.y * a.y - b.y * b.y) + k3 * 2.0f * a.y * b.y;
    HO[4] = k1 * HB[4] + k2 * (a.y * a.z - b.y * b.z) + k3 * (a.y * b.z + b.y * a.z);
    HO[5] = k1 * HB[5] + k2 * (a.z * a.z - b.z * b.z) + k3 * 2.0f * a.z * b.z;
    // ---- phase function along the direction from the cell centroid to x
    float fv, gf[3] = {0.f, 0.f, 0.f}, Hf[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    if (g == 0.0f) {
        fv = 0.25f / VRC_PI_F;
    } else {
        hg_dx((r[0] + r[1] + r[2]) * (-1.0f / 3.0f), wo, g, fv, gf, Hf);
    }
    // ---- reduced radiance at the tied furthest vertices, product rule, RGB scatter
    float inv_m = 1.0f / (float)((int)far0 + (int)far1 + (int)far2);
    float HY[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        bool fq = q == 0 ? far0 : (q == 1 ? far1 : far2);
        if (!fq) continue;
        float ir = 1.0f / rho[q];
        float3 u = r[q] * ir;
        float T = __expf(-sigma_t * rho[q]);
        float st_T = sigma_t * T;
        float3 gT = u * st_T;                              // grad T = sigma_t T (y - x)/|y - x|
        float h1 = st_T * (ir + sigma_t), h0 = -st_T * ir; // H T = st T [(1/rho + st) u u^T - I/rho]
        float HT[6] = {h1 * u.x * u.x + h0, h1 * u.x * u.y, h1 * u.x * u.z,
                       h1 * u.y * u.y + h0, h1 * u.y * u.z, h1 * u.z * u.z + h0};
        if (LOG && ((open_mask >> q) & 1u) && g != 0.0f) {
            // the light's direction of travel at the vertex y = x + r_q, and the vertex's
            // phase toward x (w = x - y = -r_q) with its x-derivatives, divided by its value
            float3 lp = r[q] + xl;
            lp = lp * rsqrtf(dot3(lp, lp));
            float fu, gu[3], Hu[6];
            hg_dx(r[q] * -1.0f, lp, g, fu, gu, Hu);
            const float ifu = 1.0f / fu;
            float gTa0[3] = {gT.x, gT.y, gT.z};
#pragma unroll
            for (int e = 0; e < 3; ++e) gu[e] *= ifu;
            const int ia[6] = {0, 0, 0, 1, 1, 2}, ja[6] = {0, 1, 2, 1, 2, 2};
#pragma unroll
            for (int e = 0; e < 6; ++e)
                HT[e] += gTa0[ia[e]] * gu[ja[e]] + gu[ia[e]] * gTa0[ja[e]] + T * Hu[e] * ifu;
            gT = f3(gT.x + T * gu[0], gT.y + T * gu[1], gT.z + T * gu[2]);
        }
        // P = Omega T
        float P = Om * T;
        float gP[3] = {T * gO.x + Om * gT.x, T * gO.y + Om * gT.y, T * gO.z + Om * gT.z};
        float gOa[3] = {gO.x, gO.y, gO.z}, gTa[3] = {gT.x, gT.y, gT.z};
        float HP[6];
        const int ii[6] = {0, 0, 0, 1, 1, 2}, jj[6] = {0, 1, 2, 1, 2, 2};
#pragma unroll
        for (int e = 0; e < 6; ++e)
            HP[e] = T * HO[e] + gTa[ii[e]] * gOa[jj[e]] + gOa[ii[e]] * gTa[jj[e]] + Om * HT[e];
        // G = f P
        float G = fv * P;
        float gG[3], HG[6];
#pragma unroll
        for (int e = 0; e < 3; ++e) gG[e] = P * gf[e] + fv * gP[e];
#pragma unroll
        for (int e = 0; e < 6; ++e)
            HG[e] = P * Hf[e] + gP[ii[e]] * gf[jj[e]] + gf[ii[e]] * gP[jj[e]] + fv * HP[e];
        float3 L = Lo[q] * inv_m;
        float Lc[3] = {L.x, L.y, L.z};
#pragma unroll
        for (int ch = 0; ch < 3; ++ch) {
            v[ch] = fmaf(Lc[ch], G, v[ch]);
#pragma unroll
            for (int e = 0; e < 3; ++e) v[3 + 3 * ch + e] = fmaf(Lc[ch], gG[e], v[3 + 3 * ch + e]);
#pragma unroll
            for (int e = 0; e < 6; ++e) v[12 + 6 * ch + e] = fmaf(Lc[ch], HG[e], v[12 + 6 * ch + e]);
        }
        float Y = 0.2126f * L.x + 0.7152f * L.y + 0.0722f * L.z;
#pragma unroll
        for (int e = 0; e < 6; ++e) HY[e] = fmaf(Y, HG[e], HY[e]);
    }
    v[30] = sqrtf(HY[0] * HY[0] + HY[3] * HY[3] + HY[5] * HY[5] +
                  2.0f * (HY[1] * HY[1] + HY[2] * HY[2] + HY[4] * HY[4]));
    return (int)far0 + (int)far1 + (int)far2;
}

// ----------------------------------------------------------------- FP64 eigenvalues
// Symmetric 3x3 eigenvalues by the trigonometric closed form (Smith, CACM 1961).
__device__ void eig3_sym(const double h[6], double lam[3]) {
    double a00 = h[0], a01 = h[1], a02 = h[2], a11 = h[3], a12 = h[4], a22 = h[5];
    double p1 = a01 * a01 + a02 * a02 + a12 * a12;
    double q = (a00 + a11 + a22) / 3.0;
    double p2 = (a00 - q) * (a00 - q) + (a11 - q) * (a11 - q) + (a22 - q) * (a22 - q) + 2.0 * p1;
    if (p2 <= 0.0) {
        lam[0] = lam[1] = lam[2] = q;
        return;
    }
    double p = sqrt(p2 / 6.0);
    double ip = 1.0 / p;
    double b00 = (a00 - q) * ip, b11 = (a11 - q) * ip, b22 = (a22 - q) * ip;
    double b01 = a01 * ip, b02 = a02 * ip, b12 = a12 * ip;
    double det = b00 * (b11 * b22 - b12 * b12) - b01 * (b01 * b22 - b12 * b02) + b02 * (b01 * b12 - b11 * b02);
    double rr = fmin(1.0, fmax(-1.0, 0.5 * det));
    double phi = acos(rr) / 3.0;
    double e1 = q + 2.0 * p * cos(phi);
    double e3 = q + 2.0 * p * cos(phi + 2.0943951023931954923);
    double e2 = 3.0 * q - e1 - e3;
    lam[0] = e3;
    lam[1] = e2;
    lam[2] = e1;
    if (lam[1] < lam[0]) { double tt = lam[0]; lam[0] = lam[1]; lam[1] = tt; }
    if (lam[2] < lam[1]) { double tt = lam[1]; lam[1] = lam[2]; lam[2] = tt; }
    if (lam[1] < lam[0]) { double tt = lam[0]; lam[0] = lam[1]; lam[1] = tt; }
}

// ----------------------------------------------------------------- FP64 eigenvectors
// Unit vector spanning the null space of the symmetric A - l I: the longest cross product
// of two of its rows (for a simple eigenvalue the rows span the plane orthogonal to the
// eigenvector).  false when every cross product vanishes (A = l I).
__device__ bool null_direction(const double h[6], double l, double v[3]) {
    const double r[3][3] = {{h[0] - l, h[1], h[2]}, {h[1], h[3] - l, h[4]}, {h[2], h[4], h[5] - l}};
    double best = 0.0;
#pragma unroll
    for (int p = 0; p < 3; ++p) {
        const double* u = r[p == 2 ? 1 : 0];
        const double* w = r[p == 0 ? 1 : 2];
        double c[3] = {u[1] * w[2] - u[2] * w[1], u[2] * w[0] - u[0] * w[2], u[0] * w[1] - u[1] * w[0]};
        double n2 = c[0] * c[0] + c[1] * c[1] + c[2] * c[2];
        if (n2 > best) {
            best = n2;
            v[0] = c[0]; v[1] = c[1]; v[2] = c[2];
        }
    }
    if (!(best > 0.0) || !isfinite(best)) return false;
    double s = 1.0 / sqrt(best);
    v[0] *= s; v[1] *= s; v[2] *= s;
    return true;
}

// Eigenvectors for the ascending eigenvalues lam (rows of V).  The eigenvalue farther from
// the middle one is isolated first by null_direction; the other two come from the 2x2
// restriction of A to the orthogonal plane, diagonalised by one plane rotation.
__device__ void eigvec3_sym(const double h[6], const double lam[3], double V[3][3]) {
    int first = (lam[2] - lam[1] >= lam[1] - lam[0]) ? 2 : 0;
    double v[3];
    if (!null_direction(h, lam[first], v)) {
        for (int i = 0; i < 3; ++i)
            for (int k = 0; k < 3; ++k) V[i][k] = i == k ? 1.0 : 0.0;
        return;
    }
    // orthonormal (u, w) spanning the plane orthogonal to v
    int m = fabs(v[0]) <= fabs(v[1]) ? (fabs(v[0]) <= fabs(v[2]) ? 0 : 2) : (fabs(v[1]) <= fabs(v[2]) ? 1 : 2);
    double e[3] = {m == 0 ? 1.0 : 0.0, m == 1 ? 1.0 : 0.0, m == 2 ? 1.0 : 0.0};
    double u[3] = {v[1] * e[2] - v[2] * e[1], v[2] * e[0] - v[0] * e[2], v[0] * e[1] - v[1] * e[0]};
    double un = 1.0 / sqrt(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
    u[0] *= un; u[1] *= un; u[2] *= un;
    double w[3] = {v[1] * u[2] - v[2] * u[1], v[2] * u[0] - v[0] * u[2], v[0] * u[1] - v[1] * u[0]};
    double Au[3] = {h[0] * u[0] + h[1] * u[1] + h[2] * u[2], h[1] * u[0] + h[3] * u[1] + h[4] * u[2],
                    h[2] * u[0] + h[4] * u[1] + h[5] * u[2]};
    double Aw[3] = {h[0] * w[0] + h[1] * w[1] + h[2] * w[2], h[1] * w[0] + h[3] * w[1] + h[4] * w[2],
                    h[2] * w[0] + h[4] * w[1] + h[5] * w[2]};
    double a = u[0] * Au[0] + u[1] * Au[1] + u[2] * Au[2];
    double b = u[0] * Aw[0] + u[1] * Aw[1] + u[2] * Aw[2];
    double c = w[0] * Aw[0] + w[1] * Aw[1] + w[2] * Aw[2];
    // (cos t, sin t) in the (u, w) frame is the eigenvector of the larger eigenvalue of
    // [[a, b], [b, c]] for t = atan2(2b, a - c) / 2
    double t = 0.5 * atan2(2.0 * b, a - c);
    double cs = cos(t), sn = sin(t);
    int hi = first == 2 ? 1 : 2, lo = first == 2 ? 0 : 1;
    for (int k = 0; k < 3; ++k) {
        V[first][k] = v[k];
        V[hi][k] = cs * u[k] + sn * w[k];
        V[lo][k] = -sn * u[k] + cs * w[k];
    }
}

// Ellipsoidal record (Eq. radiusAniso3D per eigenvalue): principal radii along the
// luminance Hessian's eigenvectors, with the clamps of the isotropic radius.
__device__ __noinline__ void write_ellipsoid(const double h[6], const double lam[3], double LY, bool bad, double eps,
                                             double r_min, double r_max, float* radii, float* axes) {
    double V[3][3];
    if (bad) {
        for (int i = 0; i < 3; ++i)
            for (int k = 0; k < 3; ++k) V[i][k] = i == k ? 1.0 : 0.0;
    } else {
        eigvec3_sym(h, lam, V);
    }
    for (int i = 0; i < 3; ++i) {
        double al = fabs(lam[i]), R;
        if (bad) R = r_min;
        else if (!(LY > 0.0)) R = r_min;
        else if (al == 0.0) R = r_max;
        else R = fmin(r_max, fmax(r_min, pow(15.0 * LY * eps / (4.0 * 3.14159265358979323846 * al), 0.2)));
        if (radii) radii[i] = (float)R;
        if (axes)
            for (int k = 0; k < 3; ++k) axes[3 * i + k] = (float)V[i][k];
    }
}

// debug output: vertex gv of shell k of record rec has radiance (the visibility decisions)
__device__ __forceinline__ void dbg_set_lit(const vrc_records_view& o, int rec, int k, int gv) {
    if (k >= o.dbg_shells) return;
    const int words = (o.dbg_stride + 31) >> 5;
    atomicOr(&o.dbg_lit[((size_t)rec * o.dbg_shells + k) * words + (gv >> 5)], 1u << (gv & 31));
}

// ----------------------------------------------------------------- the kernel
// Registers are capped at 85 per thread: 24 warps per SM, as 3 blocks of 256 (band chunks
// sized so three blocks' shared memory fits) or 2 blocks of 384 (a whole ray set that fits
// two blocks).  The cell arithmetic spills a little at this cap, but the extra warps hide the
// latency of the rest: measured 7 % faster on the mid workload and 11 % on the render one
// than 2 blocks of 256 at 128 registers.
#ifndef VRC_RECORDS_REGS
#define VRC_RECORDS_REGS 85
#endif

template <int NT, bool LOG = false>
__global__ void __launch_bounds__(NT, 65536 / (NT * VRC_RECORDS_REGS)) k_records(DevScene sc, RecArgs a) {
    constexpr int NW = NT / 32;
    extern __shared__ float4 smem4[];
    float4* ray = smem4;                                     // (d, t_end) per chunk vertex
    float* Lr = reinterpret_cast<float*>(ray + a.cap);       // [2][3][cap] vertex radiance, double-buffered
    float* Lg = Lr + a.cap;
    float* Lb = Lg + a.cap;
    float* red = Lr + 6 * a.cap;                             // [NW][32][4]
    float* mcs = red + NW * 32 * 4;                          // [NW][12]
    float* tot = mcs + NW * 12;                              // [128]
    int* misc = reinterpret_cast<int*>(tot + 128);           // [4]
    int* wq = misc + 4;                                      // [NW][64] lit-cell queues
    const int LW = ((a.cap + 31) >> 5) + 1;                  // + 1: 32-bit windows may read one word past
    unsigned* litm = reinterpret_cast<unsigned*>(wq + NW * 64);   // [2][LW]: vertex has radiance (bit per vertex)
    int* wcnt = reinterpret_cast<int*>(litm + 2 * LW);            // [NW] leftover lit cells per warp
    float* bmax = reinterpret_cast<float*>(wcnt + NW);            // [LW] furthest ray end per 32 vertices
    float* bmc = bmax + LW;                                       // [LW][3] a batch's Monte Carlo sum
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const float sigma_t = sc.sigma_t, g = sc.g;
    __shared__ int s_rec, s_item;

    for (;;) {
        if (tid == 0) {
            int item = a.item_base + atomicAdd(a.counter, 1);
            s_item = item;
            s_rec = item < a.item_end ? (a.order ? a.order[item] : item) : a.n;
        }
        __syncthreads();
        const int rec = s_rec;
        if (rec >= a.n) break;
        const int slot = s_item - a.item_base;           // pre-pass slot of this record
        const int nb = a.n_bands ? a.n_bands[rec] : a.nb0;
        if (a.n_bands && (nb < 2 || nb > a.nb0)) {
            // a per-record band count outside [2, params n_bands] would overrun the shared
            // buffers sized for params n_bands: the record is skipped and flagged
            const vrc_records_view& o = a.out;
            if (tid < 3) {
                o.L[3 * rec + tid] = 0.f;
                if (o.L_ss) o.L_ss[3 * rec + tid] = 0.f;
                if (o.L_ms) o.L_ms[3 * rec + tid] = 0.f;
                if (o.L_ff) o.L_ff[3 * rec + tid] = 0.f;
            }
            if (tid < 9) {
                o.grad[9 * rec + tid] = 0.f;
                if (o.grad_ss) o.grad_ss[9 * rec + tid] = 0.f;
                if (o.grad_ms) o.grad_ms[9 * rec + tid] = 0.f;
            }
            if (tid < 18) {
                o.hess[18 * rec + tid] = 0.f;
                if (o.hess_ss) o.hess_ss[18 * rec + tid] = 0.f;
                if (o.hess_ms) o.hess_ms[18 * rec + tid] = 0.f;
            }
            if (tid == 0 && o.kappa) o.kappa[rec] = 0.f;
            if (tid < 3) o.pos[3 * rec + tid] = a.pos[3 * rec + tid];
            if (tid == 0) {
                o.status[rec] = VRC_REC_BAD_COUNT;
                if (o.n_cells) o.n_cells[rec] = 0;
                if (o.n_far) o.n_far[rec] = 0;
                if (o.n_shells) o.n_shells[rec] = 0;
            }
            __syncthreads();
            continue;
        }
        const int ns = a.n_bands ? 2 * nb : a.ns0;
        const int N = nb * ns;
        // floor(n / ns) = umulhi(n, ns_m) for every n, ns below 2^16 (vertex and cell indices
        // of a chunk stay below its shared-memory capacity)
        const unsigned ns_m = 0xFFFFFFFFu / (unsigned)ns + 1u;
        const long long rid = a.rec_base + rec;
        const float3 x = f3(a.pos[3 * rec], a.pos[3 * rec + 1], a.pos[3 * rec + 2]);
        const float wmc = 4.0f * VRC_PI_F / (float)N;
        float acc_s = 0.f, cmp_s = 0.f, acc_m = 0.f, cmp_m = 0.f;     // lane-owned cell sums
        float mc[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f}, mcc[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        int kmax_rec = 0;
        int lit_cells = 0, far_evals = 0;                    // each lane counts its own cells
        const int CB = a.chunk_bands < nb ? a.chunk_bands : nb;

        for (int r0 = 0; r0 < nb; r0 += CB) {
            const int r1 = min(r0 + CB, nb);               // owned rows [r0, r1)
            const int r1e = min(r1, nb - 1);               // plus the next row (borrowed)
            const int rows = r1e - r0 + 1;
            const bool north = r0 == 0, south = r1 == nb;
            const int nvert = rows * ns + 2;
            const int PN = rows * ns, PS = rows * ns + 1;
            if (tid == 0) {
                misc[0] = 0;
                misc[2] = 0;
            }
            __syncthreads();
            // ---------------- primary phase
            float tmax_loc = 0.f;
            const int nvround = (nvert + 31) & ~31;
            for (int vb = warp * 32; vb < nvround; vb += NT) {
                const int lv = vb + lane;
                bool lit_v = false;
                float te_b = 0.f;
                if (lv < nvert) {
                const bool pole = lv >= rows * ns;
                const int gv = !pole ? r0 * ns + lv : (lv == PN ? N : N + 1);
                float3 d, Lo = f3(0.f, 0.f, 0.f);
                float te;
                int prim = -1;
                if (a.pre_ray) {
                    // traced by k_primary: an escaped ray has zero radiance, so its Monte
                    // Carlo term below adds an exact zero
                    const size_t gi = (size_t)slot * (size_t)a.pre_stride + gv;
                    float4 rv = __ldg(&a.pre_ray[gi]);
                    d = f3(rv.x, rv.y, rv.z);
                    te = rv.w;
                    Lo = f3(__ldg(&a.pre_Lo[3 * gi]), __ldg(&a.pre_Lo[3 * gi + 1]), __ldg(&a.pre_Lo[3 * gi + 2]));
                    prim = 0;
                } else {
                    d = ray_direction_dev(a.seed, rid, gv, nb, ns);
                    float th;
                    prim = bvh_trace<false>(sc, x, d, VRC_TMIN, 3.0e38f, &th);
                    if (prim >= 0) {
                        te = th;
                        if (a.parts != 2) Lo = surface_radiance(sc, prim, x + d * te, d);
                    } else {
                        te = cube_exit_dev(x, d);
                    }
                }
                ray[lv] = make_float4(d.x, d.y, d.z, te);
                Lr[lv] = Lo.x;
                Lg[lv] = Lo.y;
                Lb[lv] = Lo.z;
                lit_v = Lo.x != 0.f || Lo.y != 0.f || Lo.z != 0.f;
                tmax_loc = fmaxf(tmax_loc, te);
                te_b = te;
                const bool owned = lv < (r1 - r0) * ns;        // a vertex of the rows this chunk owns
                if (a.out.dbg_lit && lit_v && (owned || (pole && ((lv == PN && north) || (lv == PS && south)))))
                    dbg_set_lit(a.out, rec, 0, gv);
                if (owned && prim >= 0) {
                    float w = wmc * hg_dev(-dot3(d, a.wo), g) * __expf(-sigma_t * te);
                    neumaier(mc[0], mcc[0], w * Lo.x);
                    neumaier(mc[1], mcc[1], w * Lo.y);
                    neumaier(mc[2], mcc[2], w * Lo.z);
                }
                if (a.out.hit_prim && !a.pre_ray && (owned || (pole && ((lv == PN && north) || (lv == PS && south))))) {
                    size_t o = (size_t)rec * a.out.dbg_stride + gv;
                    a.out.hit_prim[o] = prim;
                    a.out.hit_t[o] = te;
                }
            }
                unsigned lmk = __ballot_sync(0xffffffffu, lit_v);
#pragma unroll
                for (int o = 16; o >= 1; o >>= 1) te_b = fmaxf(te_b, __shfl_xor_sync(0xffffffffu, te_b, o));
                if (lane == 0) {
                    litm[vb >> 5] = lmk;
                    bmax[vb >> 5] = te_b;
                }
            }
            atomicMax(&misc[0], __float_as_int(tmax_loc));   // non-negative floats order as ints
            __syncthreads();
            const int K = a.parts == 1 ? 0 : (int)ceilf(__int_as_float(misc[0]) / a.dt);
            kmax_rec = max(kmax_rec, K);
            // cells of this chunk
            const int nq = r1e - r0;                         // quad bands with upper row in [r0, r1e)
            const int ncell = (north ? ns : 0) + 2 * ns * nq + (south ? ns : 0);
            // Shell k's cell phase reads radiance buffer k & 1 while the same interval computes
            // shell k + 1's vertex radiance into the other buffer, and the shadow-ray latency of
            // some warps overlaps the cell arithmetic of others.
            for (int k = 0; k <= K; ++k) {
                const float tk = ((float)k - 0.5f) * a.dt;
                const float* Lrk = Lr + (k & 1) * (3 * a.cap);
                const float* Lgk = Lrk + a.cap;
                const float* Lbk = Lgk + a.cap;
                // ---------------- cell phase of shell k: lit cells are compacted into a
                // per-warp queue so cell_eval runs with all 32 lanes busy
                auto cell_verts = [&](int cc, int (&vi)[3]) {
                    if (north && cc < ns) {
                        vi[0] = PN; vi[1] = cc; vi[2] = cc + 1 == ns ? 0 : cc + 1;
                        return;
                    }
                    if (north) cc -= ns;
                    if (cc < 2 * ns * nq) {
                        int qd = cc >> 1, ri = (int)__umulhi((unsigned)qd, ns_m), j = qd - ri * ns;
                        int j1 = j + 1 == ns ? 0 : j + 1;
                        int v00 = ri * ns + j, v01 = ri * ns + j1, v10 = (ri + 1) * ns + j, v11 = (ri + 1) * ns + j1;
                        if ((cc & 1) == 0) { vi[0] = v00; vi[1] = v10; vi[2] = v11; }
                        else { vi[0] = v00; vi[1] = v11; vi[2] = v01; }
                        return;
                    }
                    cc -= 2 * ns * nq;
                    int rl = (nb - 1 - r0) * ns;
                    vi[0] = PS; vi[1] = rl + (cc + 1 == ns ? 0 : cc + 1); vi[2] = rl + cc;
                };
                auto process = [&](int c) {
                    float v[32];
#pragma unroll
                    for (int e = 0; e < 32; ++e) v[e] = 0.f;
                    int m = 0;
                    if (c >= 0) {
                        int vi[3];
                        cell_verts(c, vi);
                        float3 rr[3], Lo[3];
                        float tt[3];
                        unsigned open_mask = 0u;
#pragma unroll
                        for (int q = 0; q < 3; ++q) {
                            float4 rv = ray[vi[q]];
                            const bool open = k > 0 && tk < rv.w;
                            float tq = open ? tk : rv.w;
                            open_mask |= (unsigned)open << q;
                            tt[q] = tq;
                            rr[q] = f3(rv.x * tq, rv.y * tq, rv.z * tq);
                            Lo[q] = f3(Lrk[vi[q]], Lgk[vi[q]], Lbk[vi[q]]);
                        }
                        m = cell_eval<LOG>(rr, tt, Lo, sigma_t, g, a.wo, a.ff_signed, v, x - sc.lpos[0], open_mask);
                    }
                    lit_cells += m > 0 ? 1 : 0;
                    far_evals += m;
                    float mine = warp_transpose_reduce(v, lane);
                    if (k == 0) neumaier(acc_s, cmp_s, mine);
                    else neumaier(acc_m, cmp_m, mine);
                };
                int* wqw = wq + warp * 64;
                int qn = 0, qb = 0;                      // queue length; its first slot
                const unsigned* lmk = litm + (k & 1) * LW;
                // appends the lanes' lit cells to the warp's queue; a full queue (or a flush)
                // runs cell_eval
                auto push = [&](int c, bool lit, bool flush) {
                    unsigned msk = __ballot_sync(0xffffffffu, lit);
                    if (lit) wqw[qb + qn + __popc(msk & ((1u << lane) - 1u))] = c;
                    qn += __popc(msk);
                    __syncwarp();
                    if (qn >= 32 || (flush && qn > 0)) {
                        process(lane < qn ? wqw[qb + lane] : -1);
                        __syncwarp();
                        if (lane < qn - 32) wqw[qb + lane] = wqw[qb + lane + 32];
                        __syncwarp();
                        qn = qn > 32 ? qn - 32 : 0;
                    }
                };
                // One loop, one push site (cell_eval is inlined once).  Surface shell: a cell
                // contributes iff one of its furthest vertices (the largest ray parameter, ties
                // included) has radiance; each lane tests one cell per step.  Medium shell: a
                // vertex has radiance only while its ray is still open (t_k < t_end), and then
                // it sits at t_k, the furthest any vertex of a cell can be, so a cell
                // contributes iff one of its vertex bits is set.  Those cells are found 32 at a
                // time by word operations on the bit rows: a segment is 32 bins of one quad row
                // (its even and odd cells) or of a pole fan, segment s goes to lane s / NW of
                // warp s % NW, and each step hands the warp's next 32 lit cells to its lanes.
                const int SEG = (ns + 31) >> 5;
                const int nseg = k == 0 ? 0 : (north ? SEG : 0) + nq * SEG + (south ? SEG : 0);
                const int nround = (k != 0 || a.parts == 2) ? 0 : (ncell + 31) & ~31;   // MS cache: no surface shell
                // bits [pos, pos + 32) of the vertex mask
                auto win = [&](int pos) -> unsigned {
                    const int w = pos >> 5;
                    return __funnelshift_r(lmk[w], lmk[w + 1], pos & 31);
                };
                int base = warp * 32;                    // surface shell: next cell batch
                int sb = 0, rb0 = 0, T = 0, excl = 0;    // medium shells: segment pass, step, lit count
                unsigned me = 0u, mo = 0u;               // this lane's lit even / odd cells (fans: me)
                int cb0 = 0, cstep = 1;                  // cell of bit p: cb0 + cstep p (+ 1 if odd)
                int src = -1;                            // pass 1: this lane's merged leftover cell
                bool merged = false;
                // pass 0 scans the shell; pass 1 runs the warp's share of the merged leftovers
                // through the same push (one call site, so cell_eval is inlined once)
#pragma unroll 1
                for (int pass = 0; pass < 2; ++pass) {
                for (;;) {
                    int c = -1;
                    bool lit = false;
                    if (pass == 1) {
                        if (merged) break;
                        merged = true;
                        c = src;
                        lit = src >= 0;
                    } else if (k == 0) {
                        if (base >= nround) break;
                        c = base + lane;
                        base += NT;
                        int vi[3];
                        bool any = false;
                        if (c < ncell) {
                            cell_verts(c, vi);
#pragma unroll
                            for (int q = 0; q < 3; ++q) any |= ((lmk[vi[q] >> 5] >> (vi[q] & 31)) & 1u) != 0u;
                        }
                        if (any) {
                            float tq[3];
#pragma unroll
                            for (int q = 0; q < 3; ++q) tq[q] = ray[vi[q]].w;
                            float tmx = fmaxf(tq[0], fmaxf(tq[1], tq[2]));
#pragma unroll
                            for (int q = 0; q < 3; ++q)
                                if (tq[q] == tmx && (Lrk[vi[q]] != 0.f || Lgk[vi[q]] != 0.f || Lbk[vi[q]] != 0.f))
                                    lit = true;
                        }
                    } else {
                        if (rb0 >= T) {
                            // next segment pass: this lane's segment, its lit masks, the prefix
                            if (sb >= nseg) break;
                            const int sg = sb + lane * NW + warp;
                            sb += NT;
                            me = 0u;
                            mo = 0u;
                            cb0 = 0;
                            cstep = 1;
                            if (sg < nseg) {
                                int t = sg, kind, ri = 0, jb;
                                if (north && t < SEG) {
                                    kind = 0;
                                    jb = t;
                                } else {
                                    if (north) t -= SEG;
                                    if (t < nq * SEG) {
                                        kind = 1;
                                        ri = t / SEG;
                                        jb = t - ri * SEG;
                                    } else {
                                        kind = 2;
                                        jb = t - nq * SEG;
                                    }
                                }
                                const int j0 = jb << 5, nv = min(32, ns - j0);
                                const unsigned valid = nv == 32 ? 0xffffffffu : (1u << nv) - 1u;
                                const unsigned wb = (j0 + nv == ns) ? 1u << (nv - 1) : 0u;   // bin ns - 1: next is bin 0
                                // bins j and j + 1 (cyclic) of local vertex row rb
                                auto row = [&](int rb, unsigned& R, unsigned& Rn) {
                                    R = win(rb + j0);
                                    Rn = win(rb + j0 + 1);
                                    if (wb) Rn = ((lmk[rb >> 5] >> (rb & 31)) & 1u) ? (Rn | wb) : (Rn & ~wb);
                                };
                                if (kind == 1) {
                                    unsigned R0, R0n, R1, R1n;
                                    row(ri * ns, R0, R0n);
                                    row((ri + 1) * ns, R1, R1n);
                                    me = (R0 | R1 | R1n) & valid;        // (v00, v10, v11)
                                    mo = (R0 | R1n | R0n) & valid;       // (v00, v11, v01)
                                    cb0 = (north ? ns : 0) + 2 * (ri * ns + j0);
                                    cstep = 2;
                                } else {
                                    const int pole = kind == 0 ? PN : PS;
                                    unsigned R, Rn;
                                    row(kind == 0 ? 0 : (nb - 1 - r0) * ns, R, Rn);
                                    me = (((lmk[pole >> 5] >> (pole & 31)) & 1u) ? 0xffffffffu : (R | Rn)) & valid;
                                    cb0 = kind == 0 ? j0 : (north ? ns : 0) + 2 * ns * nq + j0;
                                }
                            }
                            const int cnt = __popc(me) + __popc(mo);
                            int incl = cnt;
#pragma unroll
                            for (int o = 1; o < 32; o <<= 1) {
                                const int y = __shfl_up_sync(0xffffffffu, incl, o);
                                if (lane >= o) incl += y;
                            }
                            excl = incl - cnt;
                            T = __shfl_sync(0xffffffffu, incl, 31);
                            rb0 = 0;
                            if (T == 0) continue;
                        }
                        // lane t of this step takes the warp's (rb0 + t)-th lit cell: its
                        // source lane by a binary search over the exclusive prefix, then the
                        // rank's bit in that lane's even mask, else in its odd mask
                        const int t = rb0 + lane;
                        rb0 += 32;
                        int src = 0;
#pragma unroll
                        for (int st = 16; st >= 1; st >>= 1) {
                            const int e = __shfl_sync(0xffffffffu, excl, src + st);
                            if (e <= t) src += st;
                        }
                        const unsigned sme = __shfl_sync(0xffffffffu, me, src);
                        const unsigned smo = __shfl_sync(0xffffffffu, mo, src);
                        const int scb = __shfl_sync(0xffffffffu, cb0, src);
                        const int sst = __shfl_sync(0xffffffffu, cstep, src);
                        int r = t - __shfl_sync(0xffffffffu, excl, src);
                        if (t < T) {
                            const int ne = __popc(sme);
                            const bool odd = r >= ne;
                            unsigned m = odd ? smo : sme;
                            if (odd) r -= ne;
                            int pbit = 0;                 // position of the r-th set bit of m
#pragma unroll
                            for (int wdt = 16; wdt >= 1; wdt >>= 1) {
                                const int lo = __popc(m & ((1u << wdt) - 1u));
                                if (r >= lo) {
                                    r -= lo;
                                    m >>= wdt;
                                    pbit += wdt;
                                }
                            }
                            c = scb + sst * pbit + (odd ? 1 : 0);
                            lit = true;
                        }
                    }
                    push(c, lit, pass == 1);
                }
                if (pass == 1) break;
                if (k + 1 <= K) {
                    // ---------------- vertex phase of medium shell k + 1, after this shell's
                    // scan: batches of 32 vertices handed out by a counter, so the warps that
                    // ran no cell batches take more of them (each vertex's radiance does not
                    // depend on who computes it, and each batch's Monte Carlo sum is taken in
                    // a fixed lane order and added after the barrier in batch order)
                    const float tn = ((float)(k + 1) - 0.5f) * a.dt;
                    const float wsh = wmc * __expf(-sigma_t * tn);
                    float* Lrn = Lr + ((k + 1) & 1) * (3 * a.cap);
                    unsigned* litn = litm + ((k + 1) & 1) * LW;
                    const int nbat = (nvert + 31) >> 5;
                    for (;;) {
                        int vb = 0;
                        if (lane == 0) vb = atomicAdd(&misc[2], 1);
                        vb = __shfl_sync(0xffffffffu, vb, 0);
                        if (vb >= nbat) break;
                        if (!(tn < bmax[vb])) {
                            // every ray of the batch has ended: no radiance and no bits (a cell
                            // reads the radiance of its furthest, open vertices only)
                            if (lane == 0) {
                                litn[vb] = 0u;
                                bmc[3 * vb] = bmc[3 * vb + 1] = bmc[3 * vb + 2] = 0.f;
                            }
                            continue;
                        }
                        const int lv = vb * 32 + lane;
                        bool lit_v = false;
                        float3 term = f3(0.f, 0.f, 0.f);     // Monte Carlo term of an owned vertex
                        if (lv < nvert) {
                            const float4 rv = ray[lv];
                            float3 Lo = f3(0.f, 0.f, 0.f);
                            if (tn < rv.w) {
                                Lo = medium_radiance(sc, x + f3(rv.x, rv.y, rv.z) * tn, f3(rv.x, rv.y, rv.z));
                                if (lv < (r1 - r0) * ns) term = Lo * (wsh * hg_dev(-(rv.x * a.wo.x + rv.y * a.wo.y + rv.z * a.wo.z), g));
                            }
                            Lrn[lv] = Lo.x;
                            Lrn[a.cap + lv] = Lo.y;
                            Lrn[2 * a.cap + lv] = Lo.z;
                            lit_v = Lo.x != 0.f || Lo.y != 0.f || Lo.z != 0.f;
                            if (a.out.dbg_lit && lit_v) {
                                const bool pole = lv >= rows * ns;
                                if (!pole ? lv < (r1 - r0) * ns : ((lv == PN && north) || (lv == PS && south)))
                                    dbg_set_lit(a.out, rec, k + 1, !pole ? r0 * ns + lv : (lv == PN ? N : N + 1));
                            }
                        }
                        const unsigned lmk = __ballot_sync(0xffffffffu, lit_v);
                        // the batch's Monte Carlo sum in a fixed lane order, whoever computes it
#pragma unroll
                        for (int o = 16; o >= 1; o >>= 1) {
                            term.x += __shfl_xor_sync(0xffffffffu, term.x, o);
                            term.y += __shfl_xor_sync(0xffffffffu, term.y, o);
                            term.z += __shfl_xor_sync(0xffffffffu, term.z, o);
                        }
                        if (lane == 0) {
                            litn[vb] = lmk;
                            bmc[3 * vb] = term.x;
                            bmc[3 * vb + 1] = term.y;
                            bmc[3 * vb + 2] = term.z;
                        }
                    }
                }
                // the warps' leftover lit cells (fewer than 32 each) of this shell: published,
                // then processed as one warp-major list, a full chunk of 32 per warp, instead
                // of one partly idle call per warp (the order is fixed: results stay
                // deterministic)
                if (lane == 0) wcnt[warp] = qn;
                __syncthreads();
                if (tid == 0) misc[2] = 0;                    // the next interval's vertex batches
                if (k + 1 <= K) {
                    // shell k + 1's batch sums, batch b into thread b % NT's compensated sums
                    for (int b = tid; b < ((nvert + 31) >> 5); b += NT) {
                        neumaier(mc[3], mcc[3], bmc[3 * b]);
                        neumaier(mc[4], mcc[4], bmc[3 * b + 1]);
                        neumaier(mc[5], mcc[5], bmc[3 * b + 2]);
                    }
                }
                {
                    int tot = 0;
                    const int t = warp * 32 + lane;
#pragma unroll
                    for (int w = 0; w < NW; ++w) {
                        const int cw = wcnt[w];
                        if (src < 0 && t >= tot && t < tot + cw) src = wq[w * 64 + (t - tot)];
                        tot += cw;
                    }
                    // the published leftovers (slots below 32) may still be read by other
                    // warps: the merged chunk goes through the upper half of the queue
                    qn = 0;
                    qb = 32;
                    if (warp * 32 >= tot) break;     // src -1 lanes: idle in the merged chunk
                }
                }
                __syncthreads();
            }
        }
        // ---------------- block reduction and outputs
        red[(warp * 32 + lane) * 4 + 0] = acc_s;
        red[(warp * 32 + lane) * 4 + 1] = cmp_s;
        red[(warp * 32 + lane) * 4 + 2] = acc_m;
        red[(warp * 32 + lane) * 4 + 3] = cmp_m;
#pragma unroll
        for (int e = 0; e < 6; ++e) {
            float s = mc[e] + mcc[e];
#pragma unroll
            for (int o = 16; o >= 1; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
            if (lane == 0) mcs[warp * 12 + e] = s;
        }
        if (tid == 0) { misc[1] = 0; misc[3] = 0; }
        __syncthreads();
        if (a.out.n_cells) {
#pragma unroll
            for (int o = 16; o >= 1; o >>= 1) {
                lit_cells += __shfl_xor_sync(0xffffffffu, lit_cells, o);
                far_evals += __shfl_xor_sync(0xffffffffu, far_evals, o);
            }
            if (lane == 0) {
                atomicAdd(&misc[1], lit_cells);
                atomicAdd(&misc[3], far_evals);
            }
        }
        __syncthreads();
        const float wms = sc.sigma_s * a.dt;                 // 1 / pdf of a medium shell
        if (warp == 0) {
            float s_s = 0.f, c_s = 0.f, s_m = 0.f, c_m = 0.f;
            for (int w = 0; w < NW; ++w) {
                neumaier(s_s, c_s, red[(w * 32 + lane) * 4 + 0]);
                neumaier(s_s, c_s, red[(w * 32 + lane) * 4 + 1]);
                neumaier(s_m, c_m, red[(w * 32 + lane) * 4 + 2]);
                neumaier(s_m, c_m, red[(w * 32 + lane) * 4 + 3]);
            }
            float vs = s_s + c_s, vm = (s_m + c_m) * wms;
            tot[lane] = vs + vm;        // total
            tot[32 + lane] = vs;        // surface shell
            tot[64 + lane] = vm;        // medium shells
            if (lane < 6) {
                float s = 0.f, cpn = 0.f;
                for (int w = 0; w < NW; ++w) neumaier(s, cpn, mcs[w * 12 + lane]);
                tot[96 + lane] = s + cpn;
            }
        }
        __syncthreads();
        const vrc_records_view& o = a.out;
        if (tid < 30) {
            // value index -> output slot: 0..2 L_ff, 3..11 grad [c][axis], 12..29 hess [c][6]
            float vt = tot[tid], vs = tot[32 + tid], vm = tot[64 + tid];
            if (tid < 3) {
                if (o.L_ff) o.L_ff[3 * rec + tid] = vt;
            } else if (tid < 12) {
                int e = tid - 3;
                o.grad[9 * rec + e] = vt;
                if (o.grad_ss) o.grad_ss[9 * rec + e] = vs;
                if (o.grad_ms) o.grad_ms[9 * rec + e] = vm;
            } else {
                int e = tid - 12;
                o.hess[18 * rec + e] = vt;
                if (o.hess_ss) o.hess_ss[18 * rec + e] = vs;
                if (o.hess_ms) o.hess_ms[18 * rec + e] = vm;
            }
        } else if (tid >= 32 && tid < 35) {
            int ch = tid - 32;
            float ls = tot[96 + ch], lm = tot[99 + ch] * wms;
            o.L[3 * rec + ch] = ls + lm;
            if (o.L_ss) o.L_ss[3 * rec + ch] = ls;
            if (o.L_ms) o.L_ms[3 * rec + ch] = lm;
            o.pos[3 * rec + ch] = ch == 0 ? x.x : (ch == 1 ? x.y : x.z);
        } else if (tid == 64) {
            // finiteness, degeneracy and conditioning; the radius comes from k_radius
            bool finite = true;
            for (int e = 0; e < 32; ++e)
                if (e != 30 && e != 31 && !isfinite(tot[e])) finite = false;
            for (int e = 0; e < 6; ++e)
                if (!isfinite(tot[96 + e])) finite = false;
            int status = finite ? 0 : VRC_REC_NONFINITE;
            if (tot[31] + tot[63] > 0.f) status |= VRC_REC_DEGENERATE;
            o.status[rec] = status;
            if (o.n_cells) o.n_cells[rec] = misc[1];
            if (o.n_far) o.n_far[rec] = misc[3];
            if (o.n_shells) o.n_shells[rec] = kmax_rec;
            if (o.kappa) {
                const double Y[3] = {0.2126, 0.7152, 0.0722};
                double h[6];
                for (int e = 0; e < 6; ++e)
                    h[e] = Y[0] * (double)tot[12 + e] + Y[1] * (double)tot[18 + e] + Y[2] * (double)tot[24 + e];
                double hn = sqrt(h[0] * h[0] + h[3] * h[3] + h[5] * h[5] + 2.0 * (h[1] * h[1] + h[2] * h[2] + h[4] * h[4]));
                o.kappa[rec] = (float)((double)tot[30] / hn);
            }
        }
        __syncthreads();
    }
}

size_t record_smem_bytes(int cap, int nt) {
    int nw = nt / 32;
    return (size_t)cap * 16 + (size_t)cap * 24 + (size_t)nw * 32 * 4 * 4 + (size_t)nw * 12 * 4 + 128 * 4 + 4 * 4 +
           (size_t)nw * 64 * 4 + 6 * (size_t)((cap + 31) / 32 + 1) * 4 + (size_t)nw * 4;
}

// Radius stage, one thread per record after the record kernel (its FP64 work would
// otherwise run on one thread of each block while the others wait): the Rec.709
// luminance of the stored L and Hessian, FP64 eigenvalues, the isotropic radius from
// the largest |eigenvalue| and, when asked for, the ellipsoid (Eq. radiusAniso3D).
__global__ void k_radius(RecArgs a) {
    int rec = blockIdx.x * blockDim.x + threadIdx.x;
    if (rec >= a.n) return;
    const vrc_records_view& o = a.out;
    const double Y[3] = {0.2126, 0.7152, 0.0722};
    const float* H = o.hess + 18 * (size_t)rec;
    double h[6];
    for (int e = 0; e < 6; ++e) h[e] = Y[0] * (double)H[e] + Y[1] * (double)H[6 + e] + Y[2] * (double)H[12 + e];
    double LY = Y[0] * (double)o.L[3 * rec] + Y[1] * (double)o.L[3 * rec + 1] + Y[2] * (double)o.L[3 * rec + 2];
    int status = o.status[rec];
    double lam[3];
    eig3_sym(h, lam);
    double lmax = fmax(fabs(lam[0]), fmax(fabs(lam[1]), fabs(lam[2])));
    bool bad = (status & VRC_REC_NONFINITE) || !isfinite(LY) || !isfinite(lmax);
    double R;
    if (bad) { status |= VRC_REC_NONFINITE | VRC_REC_CLAMP_LO; R = a.r_min; }
    else if (!(LY > 0.0)) { status |= VRC_REC_CLAMP_LO; R = a.r_min; }
    else if (lmax == 0.0) { status |= VRC_REC_CLAMP_HI; R = a.r_max; }
    else {
        R = pow(15.0 * LY * (double)a.eps / (4.0 * 3.14159265358979323846 * lmax), 0.2);
        if (R < a.r_min) { status |= VRC_REC_CLAMP_LO; R = a.r_min; }
        if (R > a.r_max) { status |= VRC_REC_CLAMP_HI; R = a.r_max; }
    }
    o.radius[rec] = (float)R;
    if (o.log_radius) o.log_radius[rec] = (float)log(R);
    o.status[rec] = status;
    if (o.eig) {
        o.eig[3 * rec] = (float)lam[0];
        o.eig[3 * rec + 1] = (float)lam[1];
        o.eig[3 * rec + 2] = (float)lam[2];
    }
    if (o.radii || o.axes)
        write_ellipsoid(h, lam, LY, bad, (double)a.eps, (double)a.r_min, (double)a.r_max,
                        o.radii ? o.radii + 3 * rec : nullptr, o.axes ? o.axes + 9 * rec : nullptr);
}

// Primary pre-pass: one thread per (work item, ray) of the current batch, the closest hit
// and the surface radiance with its shadow rays, written for the record kernel to load.
// As a flat launch it keeps every warp slot of the SM busy; inside the record kernel the
// same traversal ran with two blocks per SM between barriers, at about half the rate.
// Slots are pre_stride rays wide (a multiple of 32); a smaller ray set leaves the rest of
// its slot unused.
// 12 blocks of 128 per SM (at most 42 registers): measured 3 % faster on a 2,048-triangle
// scene and 8 % on a 250,000-triangle one than the unconstrained 70 registers
// Closest hit along o + t d (t > VRC_TMIN) for the pre-pass: the traversal of bvh_trace with
// the inner-node and leaf steps in separate loops, so the lanes of a warp that reach a leaf
// wait for the others and the warp tests its leaves together (node and triangle order per
// ray, and so the result, are those of bvh_trace).
__device__ int bvh_closest_ww(const DevScene& sc, float3 o, float3 d, float* t_hit) {
    constexpr int DONE = (int)0x80000000;
    const float big = 1e30f;
    const float tmin = VRC_TMIN;
    float best_t = 3.0e38f;
    int best = -1;
    if (sc.n_tris == 0) {
        *t_hit = best_t;
        return -1;
    }
    const float3 inv = f3(fabsf(d.x) > 1e-30f ? 1.0f / d.x : copysignf(big, d.x),
                          fabsf(d.y) > 1e-30f ? 1.0f / d.y : copysignf(big, d.y),
                          fabsf(d.z) > 1e-30f ? 1.0f / d.z : copysignf(big, d.z));
    const float3 oi = f3(o.x * inv.x, o.y * inv.y, o.z * inv.z);
    int stack[VRC_STACK];
    int sp = 0;
    int code = 0;
    for (;;) {
        while (code >= 0) {
            const float4* N = sc.nodes + 4 * code;
            const float4 n0 = __ldg(N), n1 = __ldg(N + 1), n2 = __ldg(N + 2), n3 = __ldg(N + 3);
            float a0 = fmaf(n0.x, inv.x, -oi.x), a1 = fmaf(n0.y, inv.x, -oi.x);
            float b0 = fmaf(n0.z, inv.y, -oi.y), b1 = fmaf(n0.w, inv.y, -oi.y);
            float z0 = fmaf(n2.x, inv.z, -oi.z), z1 = fmaf(n2.y, inv.z, -oi.z);
            const float tn0 = fmaxf(fmaxf(fminf(a0, a1), fminf(b0, b1)), fmaxf(fminf(z0, z1), tmin));
            const float tf0 = fminf(fminf(fmaxf(a0, a1), fmaxf(b0, b1)), fminf(fmaxf(z0, z1), best_t));
            a0 = fmaf(n1.x, inv.x, -oi.x); a1 = fmaf(n1.y, inv.x, -oi.x);
            b0 = fmaf(n1.z, inv.y, -oi.y); b1 = fmaf(n1.w, inv.y, -oi.y);
            z0 = fmaf(n2.z, inv.z, -oi.z); z1 = fmaf(n2.w, inv.z, -oi.z);
            const float tn1 = fmaxf(fmaxf(fminf(a0, a1), fminf(b0, b1)), fmaxf(fminf(z0, z1), tmin));
            const float tf1 = fminf(fminf(fmaxf(a0, a1), fmaxf(b0, b1)), fminf(fmaxf(z0, z1), best_t));
            const bool h0 = tn0 <= tf0, h1 = tn1 <= tf1;
            const int c0 = __float_as_int(n3.x), c1 = __float_as_int(n3.y);
            if (h0 && h1) {
                const int nearc = tn0 <= tn1 ? c0 : c1, farc = tn0 <= tn1 ? c1 : c0;
                if (sp < VRC_STACK) stack[sp++] = farc;
                code = nearc;
            } else if (h0) {
                code = c0;
            } else if (h1) {
                code = c1;
            } else {
                code = sp == 0 ? DONE : stack[--sp];
            }
        }
        if (code == DONE) break;
        const int z = -code - 1;
        const int first = z >> 3, count = (z & 7) + 1;
        for (int k = first; k < first + count; ++k) {
            float t;
            int id;
            if (tri_hit(sc.tris, k, o, d, tmin, best_t * (1.0f + 1e-7f) + 1e-30f, &t, &id)) {
                if (t < best_t || (t == best_t && id < best)) {
                    best_t = t;
                    best = id;
                }
            }
        }
        code = sp == 0 ? DONE : stack[--sp];
        if (code == DONE) break;
    }
    *t_hit = best_t;
    return best;
}

// 14 blocks of 128 per SM (at most 36 registers): measured against 12 (40 registers) 0.853 ->
// 0.834 ms on the mid workload, 0.880 -> 0.874 ms on the render scene; 16 blocks no better
__global__ void __launch_bounds__(128, 14) k_primary(DevScene sc, RecArgs a, float4* ray, float* Lo_out) {
    // a batch holds at most PRE_MAX_RAYS (< 2^31) rays: 32-bit index arithmetic
    const unsigned i = blockIdx.x * blockDim.x + threadIdx.x;
    const int slot = (int)(i / (unsigned)a.pre_stride);
    int gv = (int)(i - (unsigned)slot * (unsigned)a.pre_stride);
    const int item = a.item_base + slot;
    if (item >= a.item_end) return;
    const int rec = a.order ? a.order[item] : item;
    const int nb = a.n_bands ? a.n_bands[rec] : a.nb0;
    if (a.n_bands && (nb < 2 || nb > a.nb0)) return;        // flagged by the record kernel
    const int ns = a.n_bands ? 2 * nb : a.ns0;
    if (gv >= nb * ns + 2) return;
    if (gv < nb * ns && (nb & 7) == 0 && (ns & 3) == 0) {
        // a warp (slots are a multiple of 32 rays wide) traces a tile of 8 bands x 4 bins of
        // strata, not 32 bins of one band: neighbouring directions take similar paths through
        // the BVH (measured against 4 x 8 and 2 x 16 tiles: 1-2 % and 7 % faster)
        const int tile = gv >> 5, w = gv & 31, tpr = ns >> 2;
        const int bg = tile / tpr, bt = tile - bg * tpr;
        gv = (8 * bg + (w >> 2)) * ns + 4 * bt + (w & 3);
    }
    const float3 x = f3(a.pos[3 * rec], a.pos[3 * rec + 1], a.pos[3 * rec + 2]);
    const float3 d = ray_direction_dev(a.seed, a.rec_base + rec, gv, nb, ns);
    float th;
    // measured: the separate leaf loop is 12 % faster on a 250,000-triangle scene and 0.8 %
    // slower on a 2,048-triangle one (whose traversals are short)
    const int prim = sc.n_tris > 16384 ? bvh_closest_ww(sc, x, d, &th) : bvh_trace<false>(sc, x, d, VRC_TMIN, 3.0e38f, &th);
    float3 Lo = f3(0.f, 0.f, 0.f);
    float te;
    if (prim >= 0) {
        te = th;
        if (a.parts != 2) Lo = surface_radiance(sc, prim, x + d * te, d);
    } else {
        te = cube_exit_dev(x, d);
    }
    const unsigned at = (unsigned)slot * (unsigned)a.pre_stride + (unsigned)gv;   // the ray's own place
    ray[at] = make_float4(d.x, d.y, d.z, te);
    Lo_out[3 * at] = Lo.x;
    Lo_out[3 * at + 1] = Lo.y;
    Lo_out[3 * at + 2] = Lo.z;
    if (a.out.hit_prim) {
        size_t o = (size_t)rec * a.out.dbg_stride + gv;
        a.out.hit_prim[o] = prim;
        a.out.hit_t[o] = te;
    }
}

// The event quadruple for this launch when per-kernel timing is on (NULL otherwise, when
// the stream is being captured into a graph, or when 64 launches are pending).
static cudaEvent_t* timing_slot(vrc_scene* s, cudaStream_t st) {
    if (!s->timing) return nullptr;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) return nullptr;
    if (s->n_timed >= 64) return nullptr;
    if (s->n_timed >= s->t_ev_made) {
        for (int e = 0; e < 4; ++e)
            if (cudaEventCreate(&s->t_ev[s->n_timed][e]) != cudaSuccess) return nullptr;
        s->t_ev_made = s->n_timed + 1;
    }
    return s->t_ev[s->n_timed++];
}

// Records per pre-pass batch: the pre-pass buffers hold `cap` rays of `stride`-ray slots.
static int batch_records(long long cap, int stride, int n) {
    long long b = cap / stride;
    return (int)(b < 1 ? 1 : (b > n ? n : b));
}

template <int NT, bool LOG = false>
int launch_records(vrc_scene* s, const RecArgs& a0, size_t smem, cudaStream_t st) {
    auto kfn = k_records<NT, LOG>;
    if (cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return VRC_ERR_UNSUPPORTED;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kfn, NT, smem) != cudaSuccess || per_sm < 1)
        return VRC_ERR_UNSUPPORTED;
    if (s->tuning.blocks_per_sm > 0 && s->tuning.blocks_per_sm < per_sm) per_sm = s->tuning.blocks_per_sm;
    DevScene dv = s->dev;
    dv.use_lb = s->tuning.shadow_bvh ? 0 : 1;
    RecArgs a = a0;
    // batches of work items (in `order` when given) whose ray sets fit the pre-pass buffers
    const int B = a.pre_ray ? batch_records(s->pre_cap, a.pre_stride, a.n) : a.n;
    const int n_batches = (a.n + B - 1) / B;
    cudaEvent_t* ev = n_batches == 1 ? timing_slot(s, st) : nullptr;
    if (ev) cudaEventRecord(ev[0], st);
    for (int b0 = 0; b0 < a.n; b0 += B) {
        a.item_base = b0;
        a.item_end = b0 + B < a.n ? b0 + B : a.n;
        const int nb_items = a.item_end - a.item_base;
        if (cudaMemsetAsync(s->d_counter, 0, sizeof(int), st) != cudaSuccess) return VRC_ERR_CUDA;
        if (a.pre_ray) {
            const long long rays = (long long)nb_items * a.pre_stride;
            k_primary<<<(unsigned)((rays + 127) / 128), 128, 0, st>>>(dv, a, const_cast<float4*>(a.pre_ray),
                                                                       const_cast<float*>(a.pre_Lo));
        }
        if (ev) cudaEventRecord(ev[1], st);
        int grid = per_sm * s->sm_count;
        if (grid > nb_items) grid = nb_items;
        if (grid < 1) grid = 1;
        kfn<<<grid, NT, smem, st>>>(dv, a);
    }
    if (ev) cudaEventRecord(ev[2], st);
    // one warp per block: a few thousand records then spread over every SM's FP64 units
    k_radius<<<(a.n + 31) / 32, 32, 0, st>>>(a);
    if (ev) cudaEventRecord(ev[3], st);
    return cudaGetLastError() == cudaSuccess ? VRC_OK : VRC_ERR_CUDA;
}

// Largest-first order of records with uneven ray counts (longest-processing-time
// scheduling for the persistent blocks): a counting sort by band count, descending.
// hist has 258 ints: [0, 256] bucket counts for bands 1..256, then the running offsets.
__global__ void k_lpt_hist(const int* n_bands, int n, int* hist) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) atomicAdd(&hist[256 - min(256, max(1, n_bands[i]))], 1);   // bucket 0 = most bands
}
__global__ void k_lpt_scan(int* hist) {
    if (threadIdx.x == 0) {
        int run = 0;
        for (int b = 0; b < 257; ++b) {
            int c = hist[b];
            hist[b] = run;
            run += c;
        }
    }
}
__global__ void k_lpt_scatter(const int* n_bands, int n, int* hist, int* order) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) order[atomicAdd(&hist[256 - min(256, max(1, n_bands[i]))], 1)] = i;
}

}  // namespace

static int ensure_order_scratch(vrc_scene* s, int n) {
    if (s->order_cap >= n) return VRC_OK;
    cudaFree(s->d_order);
    s->d_order = nullptr;
    s->order_cap = 0;
    if (cudaMalloc((void**)&s->d_order, sizeof(int) * ((size_t)n + 258)) != cudaSuccess) return VRC_ERR_OOM;
    s->order_cap = n;
    return VRC_OK;
}

// Primary pre-pass buffers for `rays` rays (28 B per ray), at most PRE_MAX_RAYS: larger
// launches run in batches of work items whose slots fit.
constexpr long long PRE_MAX_RAYS = 64ll << 20;   // 1.75 GB of buffers
static int ensure_pre_scratch(vrc_scene* s, long long rays) {
    if (s->pre_cap >= rays) return VRC_OK;
    cudaFree(s->d_pre_ray);
    cudaFree(s->d_pre_Lo);
    s->d_pre_ray = nullptr;
    s->d_pre_Lo = nullptr;
    s->pre_cap = 0;
    if (cudaMalloc((void**)&s->d_pre_ray, sizeof(float4) * (size_t)rays) != cudaSuccess ||
        cudaMalloc((void**)&s->d_pre_Lo, 3 * sizeof(float) * (size_t)rays) != cudaSuccess) {
        cudaFree(s->d_pre_ray);
        s->d_pre_ray = nullptr;
        return VRC_ERR_OOM;
    }
    s->pre_cap = rays;
    return VRC_OK;
}

extern "C" int vrc_set_record_tuning(vrc_scene* s, const vrc_record_tuning* t) {
    if (!s || !t) return VRC_ERR_INVALID;
    if (t->threads != 0 && t->threads != 128 && t->threads != 256 && t->threads != 384 && t->threads != 512)
        return VRC_ERR_INVALID;
    if (t->chunk_bands < 0 || t->blocks_per_sm < 0 || t->shadow_bvh < 0 || t->shadow_bvh > 1 || t->no_prepass < 0 ||
        t->no_prepass > 1)
        return VRC_ERR_INVALID;
    s->tuning = *t;
    return VRC_OK;
}

extern "C" int vrc_get_record_tuning(const vrc_scene* s, vrc_record_tuning* t) {
    if (!s || !t) return VRC_ERR_INVALID;
    *t = s->tuning;
    return VRC_OK;
}

extern "C" int vrc_record_timing(vrc_scene* s, int32_t enable) {
    if (!s || enable < 0 || enable > 1) return VRC_ERR_INVALID;
    s->timing = enable;
    s->n_timed = 0;
    return VRC_OK;
}

extern "C" int vrc_record_kernel_times(vrc_scene* s, float* ms3, int32_t* launches) {
    if (!s || !ms3) return VRC_ERR_INVALID;
    ms3[0] = ms3[1] = ms3[2] = 0.f;
    int n = s->n_timed;
    for (int i = 0; i < n; ++i) {
        if (cudaEventSynchronize(s->t_ev[i][3]) != cudaSuccess) return VRC_ERR_CUDA;
        for (int k = 0; k < 3; ++k) {
            float ms = 0.f;
            if (cudaEventElapsedTime(&ms, s->t_ev[i][k], s->t_ev[i][k + 1]) != cudaSuccess) return VRC_ERR_CUDA;
            ms3[k] += ms;
        }
    }
    if (launches) *launches = n;
    s->n_timed = 0;
    return VRC_OK;
}

extern "C" int vrc_compute_records(vrc_scene* s, const float* d_pos, int32_t n, const int32_t* d_n_bands,
                                   const vrc_record_params* p, const vrc_records_view* out, void* stream) {
    if (!s || !p || !out || n < 0) return VRC_ERR_INVALID;
    if (n == 0) return VRC_OK;
    if (!d_pos || !out->L || !out->grad || !out->hess || !out->radius || !out->status || !out->pos)
        return VRC_ERR_INVALID;
    int nb = p->n_bands, ns = d_n_bands ? 2 * p->n_bands : p->n_bins;
    if (nb < 1 || ns < 3 || !(p->dt > 0.f) || !(p->eps > 0.f) || !(p->r_min > 0.f) || !(p->r_max >= p->r_min))
        return VRC_ERR_INVALID;
    if (p->parts < 0 || p->parts > 2) return VRC_ERR_INVALID;
    if (nb > 256 || ns > 512) return VRC_ERR_UNSUPPORTED;
    if (p->lo_grad && s->dev.n_lights != 1) return VRC_ERR_UNSUPPORTED;   // one light's phase per vertex
    if (p->lo_grad && s->tuning.threads != 0 && s->tuning.threads != 256 && s->tuning.threads != 384 &&
        s->tuning.threads != 512)
        return VRC_ERR_UNSUPPORTED;                     // compiled for the default block shapes
    if ((out->hit_prim != nullptr) != (out->hit_t != nullptr)) return VRC_ERR_INVALID;
    if (out->hit_prim && out->dbg_stride < nb * ns + 2) return VRC_ERR_INVALID;
    if (out->dbg_lit && (!out->hit_prim || out->dbg_shells < 1)) return VRC_ERR_INVALID;
    cudaStream_t st = (cudaStream_t)stream;
    int nt = s->tuning.threads ? s->tuning.threads : 256;
    int cb = s->tuning.chunk_bands;
    if (!s->tuning.threads && cb <= 0 && n <= s->sm_count && record_smem_bytes((nb + 1) * ns + 2, 512) <= 200 * 1024) {
        // at most one record per SM (placement's small waves): one block of 512 threads per
        // record with the whole ray set, 16 warps on its shells instead of 12 (measured, 32 x
        // 64 rays: 4 records 0.217 -> 0.182 ms, 150 records 0.286 -> 0.243 ms; at 304 and
        // more records two blocks of 384 per SM stay faster; 768 threads: slower than 512)
        nt = 512;
        cb = nb;
    } else if (!s->tuning.threads && cb <= 0 && !p->lo_grad && n >= 6 * s->sm_count &&
        record_smem_bytes((nb + 1) * ns + 2, 128) <= 36 * 1024) {
        // small ray sets (up to about 16 x 32) and enough records to fill six blocks per SM:
        // blocks of 128 threads with the whole ray set, so that a record's few vertex and
        // cell batches keep its warps busy (measured: 8 x 16 rays, 24,777 records 3.84 ->
        // 2.11 ms; 16 x 32 rays, 4,096 records 1.02 -> 0.73 ms; 64 records stay faster at 384)
        nt = 128;
        cb = nb;
    } else if (!s->tuning.threads && cb <= 0 && record_smem_bytes((nb + 1) * ns + 2, 384) <= 110 * 1024) {
        // a whole ray set fits two blocks of 384 per SM: one chunk per record (no borrowed
        // row, half the shell barriers of two chunks); measured 2 % faster than three blocks
        // of 256 with 16-band chunks on a 32 x 64 ray set
        nt = 384;
        cb = nb;
    }
    // bands per chunk: as many as fit a shared-memory budget (three blocks per SM)
    if (cb <= 0) {
        cb = nb;
        while (cb > 1 && record_smem_bytes((cb + 1) * ns + 2, nt) > 72 * 1024) cb = (cb + 1) / 2;
    }
    if (cb > nb) cb = nb;
    int cap = (cb + 1) * ns + 2;
    size_t smem = record_smem_bytes(cap, nt);
    if (smem > 227 * 1024) return VRC_ERR_UNSUPPORTED;
    RecArgs a;
    a.pos = d_pos;
    a.n = n;
    a.n_bands = d_n_bands;
    a.nb0 = nb;
    a.ns0 = ns;
    a.dt = p->dt;
    a.eps = p->eps;
    a.wo = make_float3(p->omega_o[0], p->omega_o[1], p->omega_o[2]);
    a.seed = p->seed;
    a.ff_signed = p->ff_signed;
    a.r_min = p->r_min;
    a.r_max = p->r_max;
    a.rec_base = p->rec_base;
    a.out = *out;
    a.chunk_bands = cb;
    a.cap = cap;
    a.counter = s->d_counter;
    a.order = nullptr;
    a.parts = p->parts;
    a.lo_grad = p->lo_grad ? 1 : 0;
    a.pre_ray = nullptr;
    a.pre_Lo = nullptr;
    a.pre_stride = (nb * ns + 2 + 31) & ~31;          // the largest ray set of the launch, whole warps
    a.item_base = 0;
    a.item_end = n;
    if (!s->tuning.no_prepass) {
        long long rays = (long long)n * a.pre_stride;
        if (rays > PRE_MAX_RAYS) rays = PRE_MAX_RAYS / a.pre_stride * a.pre_stride;
        if (rays < a.pre_stride) rays = a.pre_stride;
        if (ensure_pre_scratch(s, rays) == VRC_OK) {
            a.pre_ray = s->d_pre_ray;
            a.pre_Lo = s->d_pre_Lo;
        }
    }
    if (d_n_bands && n > 1) {
        // largest ray sets first; the order and histogram live in scene-owned scratch
        int rc = ensure_order_scratch(s, n);
        if (rc != VRC_OK) return rc;
        int* hist = s->d_order + n;
        VRC_CUDA_CHECK(cudaMemsetAsync(hist, 0, sizeof(int) * 258, st));
        int nbk = (n + 255) / 256;
        k_lpt_hist<<<nbk, 256, 0, st>>>(d_n_bands, n, hist);
        k_lpt_scan<<<1, 32, 0, st>>>(hist);
        k_lpt_scatter<<<nbk, 256, 0, st>>>(d_n_bands, n, hist, s->d_order);
        a.order = s->d_order;
    }
    if (a.lo_grad)   // compiled for the default block shapes only (not the 128-thread one)
        return nt == 384 ? launch_records<384, true>(s, a, smem, st)
                         : (nt == 512 ? launch_records<512, true>(s, a, smem, st)
                                      : launch_records<256, true>(s, a, smem, st));
    switch (nt) {
        case 128: return launch_records<128>(s, a, smem, st);
        case 384: return launch_records<384>(s, a, smem, st);
        case 512: return launch_records<512>(s, a, smem, st);
        default: return launch_records<256>(s, a, smem, st);
    }
}

extern "C" int vrc_compute_records_host(vrc_scene* s, const float* h_pos, int32_t n, const vrc_record_params* p,
                                        float* h_L, float* h_grad, float* h_hess, float* h_radius,
                                        int32_t* h_status) {
    if (!s || !p || n < 0 || (n > 0 && !h_pos)) return VRC_ERR_INVALID;
    if (n == 0) return VRC_OK;
    // staging layout (floats per record): pos 3, L 3, grad 9, hess 18, radius 1, status 1, pos copy 3
    const size_t per = 38;
    size_t need = per * (size_t)n;
    if (s->h_stage_floats < need) {
        cudaFree(s->h_stage_dev);
        s->h_stage_dev = nullptr;
        s->h_stage_floats = 0;
        if (cudaMalloc((void**)&s->h_stage_dev, need * sizeof(float)) != cudaSuccess) return VRC_ERR_OOM;
        s->h_stage_floats = need;
    }
    float* base = s->h_stage_dev;
    float* d_pos = base;
    vrc_records_view v = {};
    v.L = base + 3 * (size_t)n;
    v.grad = base + 6 * (size_t)n;
    v.hess = base + 15 * (size_t)n;
    v.radius = base + 33 * (size_t)n;
    v.status = reinterpret_cast<int32_t*>(base + 34 * (size_t)n);
    v.pos = base + 35 * (size_t)n;
    VRC_CUDA_CHECK(cudaMemcpy(d_pos, h_pos, 3 * sizeof(float) * n, cudaMemcpyHostToDevice));
    int rc = vrc_compute_records(s, d_pos, n, nullptr, p, &v, nullptr);
    if (rc != VRC_OK) return rc;
    if (h_L) VRC_CUDA_CHECK(cudaMemcpy(h_L, v.L, 3 * sizeof(float) * n, cudaMemcpyDeviceToHost));
    if (h_grad) VRC_CUDA_CHECK(cudaMemcpy(h_grad, v.grad, 9 * sizeof(float) * n, cudaMemcpyDeviceToHost));
    if (h_hess) VRC_CUDA_CHECK(cudaMemcpy(h_hess, v.hess, 18 * sizeof(float) * n, cudaMemcpyDeviceToHost));
    if (h_radius) VRC_CUDA_CHECK(cudaMemcpy(h_radius, v.radius, sizeof(float) * n, cudaMemcpyDeviceToHost));
    if (h_status) VRC_CUDA_CHECK(cudaMemcpy(h_status, v.status, sizeof(int32_t) * n, cudaMemcpyDeviceToHost));
    VRC_CUDA_CHECK(cudaDeviceSynchronize());
    return VRC_OK;
}

// grow a scene-owned device staging buffer to hold `need` floats
static int stage(float** buf, size_t* have, size_t need) {
    if (*have >= need) return VRC_OK;
    cudaFree(*buf);
    *buf = nullptr;
    *have = 0;
    if (cudaMalloc((void**)buf, need * sizeof(float)) != cudaSuccess) return VRC_ERR_OOM;
    *have = need;
    return VRC_OK;
}

extern "C" int vrc_cache_step_host(vrc_scene* s, vrc_grid** grid, const float* h_pos, int32_t n,
                                   const vrc_record_params* p, const float* h_q, int32_t nq, float* h_L,
                                   float* h_grad, float* h_hess, float* h_radius, int32_t* h_status, float* h_rgb,
                                   int32_t* h_qstatus) {
    if (!s || !grid || !p || n < 0 || nq < 0 || (n > 0 && !h_pos) || (nq > 0 && (!h_q || !h_rgb || !h_qstatus)))
        return VRC_ERR_INVALID;
    if (p->extrap_order != 1 && p->extrap_order != 2) return VRC_ERR_INVALID;
    if (!s->step_made) {
        for (int i = 0; i < 2; ++i) {
            if (cudaStreamCreateWithFlags(&s->step_st[i], cudaStreamNonBlocking) != cudaSuccess ||
                cudaEventCreateWithFlags(&s->step_ev[i], cudaEventDisableTiming) != cudaSuccess)
                return VRC_ERR_CUDA;
        }
        s->step_made = 1;
    }
    // staging (floats per record): pos 3, L 3, grad 9, hess 18, radius 1, status 1, pos copy 3;
    // per query: point 3 in, rgb 3 + status 1 out
    int rc;
    if ((rc = stage(&s->h_stage_dev, &s->h_stage_floats, 38 * (size_t)(n > 0 ? n : 1))) ||
        (rc = stage(&s->q_stage_dev, &s->q_stage_floats, 7 * (size_t)(nq > 0 ? nq : 1))))
        return rc;
    cudaStream_t main = s->step_st[0], side = s->step_st[1];
    float* base = s->h_stage_dev;
    float* d_pos = base;
    vrc_records_view v = {};
    v.L = base + 3 * (size_t)n;
    v.grad = base + 6 * (size_t)n;
    v.hess = base + 15 * (size_t)n;
    v.radius = base + 33 * (size_t)n;
    v.status = reinterpret_cast<int32_t*>(base + 34 * (size_t)n);
    v.pos = base + 35 * (size_t)n;
    float* d_q = s->q_stage_dev;
    float* d_rgb = d_q + 3 * (size_t)nq;
    int32_t* d_qst = reinterpret_cast<int32_t*>(d_rgb + 3 * (size_t)nq);
    // the queries arrive on the side stream while the records are computed
    if (nq > 0) VRC_CUDA_CHECK(cudaMemcpyAsync(d_q, h_q, 3 * sizeof(float) * nq, cudaMemcpyHostToDevice, side));
    VRC_CUDA_CHECK(cudaEventRecord(s->step_ev[1], side));
    if (n > 0) {
        VRC_CUDA_CHECK(cudaMemcpyAsync(d_pos, h_pos, 3 * sizeof(float) * n, cudaMemcpyHostToDevice, main));
        if ((rc = vrc_compute_records(s, d_pos, n, nullptr, p, &v, main)) != VRC_OK) return rc;
        // the records leave on the side stream while the grid and the queries run
        VRC_CUDA_CHECK(cudaEventRecord(s->step_ev[0], main));
        VRC_CUDA_CHECK(cudaStreamWaitEvent(side, s->step_ev[0], 0));
        if (h_L) VRC_CUDA_CHECK(cudaMemcpyAsync(h_L, v.L, 3 * sizeof(float) * n, cudaMemcpyDeviceToHost, side));
        if (h_grad) VRC_CUDA_CHECK(cudaMemcpyAsync(h_grad, v.grad, 9 * sizeof(float) * n, cudaMemcpyDeviceToHost, side));
        if (h_hess) VRC_CUDA_CHECK(cudaMemcpyAsync(h_hess, v.hess, 18 * sizeof(float) * n, cudaMemcpyDeviceToHost, side));
        if (h_radius) VRC_CUDA_CHECK(cudaMemcpyAsync(h_radius, v.radius, sizeof(float) * n, cudaMemcpyDeviceToHost, side));
        if (h_status)
            VRC_CUDA_CHECK(cudaMemcpyAsync(h_status, v.status, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, side));
    }
    rc = *grid ? vrc_rebuild_record_grid(*grid, &v, n, p->extrap_order, 0, main)
               : vrc_build_record_grid(&v, n, p->extrap_order, grid, main);
    if (rc != VRC_OK) return rc;
    if (nq > 0) {
        VRC_CUDA_CHECK(cudaStreamWaitEvent(main, s->step_ev[1], 0));
        if ((rc = vrc_query_inscatter(*grid, d_q, nq, d_rgb, d_qst, main)) != VRC_OK) return rc;
        VRC_CUDA_CHECK(cudaMemcpyAsync(h_rgb, d_rgb, 3 * sizeof(float) * nq, cudaMemcpyDeviceToHost, main));
        VRC_CUDA_CHECK(cudaMemcpyAsync(h_qstatus, d_qst, sizeof(int32_t) * nq, cudaMemcpyDeviceToHost, main));
    }
    VRC_CUDA_CHECK(cudaStreamSynchronize(main));
    VRC_CUDA_CHECK(cudaStreamSynchronize(side));
    return VRC_OK;
}

// ----------------------------------------------------------------- CUDA graph
struct vrc_graph {
    cudaGraph_t graph;
    cudaGraphExec_t exec;
};

extern "C" int vrc_records_graph_create(vrc_scene* s, const float* d_pos, int32_t n, const int32_t* d_n_bands,
                                        const vrc_record_params* p, const vrc_records_view* out, vrc_graph** g) {
    if (!s || !p || !out || !g || n < 1) return VRC_ERR_INVALID;
    *g = nullptr;
    if (d_n_bands) {
        int rc = ensure_order_scratch(s, n);     // no allocation may happen inside the capture
        if (rc != VRC_OK) return rc;
    }
    if (!s->tuning.no_prepass) {
        const long long stride =
            ((d_n_bands ? 2ll * p->n_bands * p->n_bands + 2 : (long long)p->n_bands * p->n_bins + 2) + 31) & ~31ll;
        long long rays = (long long)n * stride;
        if (rays > PRE_MAX_RAYS) rays = PRE_MAX_RAYS / stride * stride;
        if (rays < stride) rays = stride;
        int rc = ensure_pre_scratch(s, rays);
        if (rc != VRC_OK) return rc;
    }
    cudaStream_t cs;
    VRC_CUDA_CHECK(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    vrc_graph* G = new vrc_graph();
    int rc = VRC_OK;
    if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess) rc = VRC_ERR_CUDA;
    if (rc == VRC_OK) {
        int rc2 = vrc_compute_records(s, d_pos, n, d_n_bands, p, out, cs);
        cudaError_t e = cudaStreamEndCapture(cs, &G->graph);
        if (rc2 != VRC_OK) rc = rc2;
        else if (e != cudaSuccess) rc = VRC_ERR_CUDA;
    }
    if (rc == VRC_OK && cudaGraphInstantiate(&G->exec, G->graph, 0) != cudaSuccess) rc = VRC_ERR_CUDA;
    cudaStreamDestroy(cs);
    if (rc != VRC_OK) {
        if (G->graph) cudaGraphDestroy(G->graph);
        delete G;
        cudaGetLastError();
        return rc;
    }
    *g = G;
    return VRC_OK;
}

extern "C" int vrc_graph_launch(vrc_graph* g, void* stream) {
    if (!g) return VRC_ERR_INVALID;
    return cudaGraphLaunch(g->exec, (cudaStream_t)stream) == cudaSuccess ? VRC_OK : VRC_ERR_CUDA;
}

extern "C" void vrc_graph_destroy(vrc_graph* g) {
    if (!g) return;
    if (g->exec) cudaGraphExecDestroy(g->exec);
    if (g->graph) cudaGraphDestroy(g->graph);
    delete g;
}

// ----------------------------------------------------------------- autotuner
namespace {
// cached winners, keyed by ray set, mixed counts, record parts, log2 of the record count
// and log2 of the scene's triangle count
struct TuneEntry {
    int nb, ns, mixed, parts, logn, logt;
    vrc_record_tuning t;
};
std::mutex g_tune_mutex;
std::vector<TuneEntry> g_tune_cache;
}  // namespace

extern "C" int vrc_autotune_records(vrc_scene* s, const float* d_pos, int32_t n, const int32_t* d_n_bands,
                                    const vrc_record_params* p, const vrc_records_view* out, void* stream,
                                    vrc_record_tuning* best) {
    if (!s || !p || !out || n < 1) return VRC_ERR_INVALID;
    int logn = 0;
    while ((1 << (logn + 1)) <= n) ++logn;
    const int mixed = d_n_bands ? 1 : 0;
    int logt = 0;
    while ((1 << (logt + 1)) <= s->n_prims) ++logt;
    {
        std::lock_guard<std::mutex> lock(g_tune_mutex);
        for (const TuneEntry& e : g_tune_cache)
            if (e.nb == p->n_bands && e.ns == p->n_bins && e.mixed == mixed && e.parts == p->parts && e.logn == logn &&
                e.logt == logt) {
                s->tuning = e.t;
                if (best) *best = e.t;
                return VRC_OK;
            }
    }
    cudaStream_t st = (cudaStream_t)stream;
    int m = n < 16384 ? n : 16384;
    vrc_record_tuning saved = s->tuning, top = saved;
    float top_ms = 3.0e38f;
    cudaEvent_t e0, e1;
    VRC_CUDA_CHECK(cudaEventCreate(&e0));
    VRC_CUDA_CHECK(cudaEventCreate(&e1));
    const int threads[4] = {128, 256, 384, 512};
    const int chunks[4] = {0, 8, 16, 32};
    const int n_pre = 2;                      // with and without the primary pre-pass
    for (int pi = 0; pi < n_pre; ++pi)
    for (int ti = 0; ti < 4; ++ti)
        for (int ci = 0; ci < 4; ++ci) {
            if (chunks[ci] > p->n_bands) continue;
            vrc_record_tuning t = saved;
            t.threads = threads[ti];
            t.chunk_bands = chunks[ci];
            t.blocks_per_sm = 0;
            t.no_prepass = pi;
            s->tuning = t;
            if (vrc_compute_records(s, d_pos, m, d_n_bands, p, out, stream) != VRC_OK) continue;
            cudaEventRecord(e0, st);
            bool ok = true;
            for (int r = 0; r < 2 && ok; ++r) ok = vrc_compute_records(s, d_pos, m, d_n_bands, p, out, stream) == VRC_OK;
            cudaEventRecord(e1, st);
            if (!ok || cudaEventSynchronize(e1) != cudaSuccess) continue;
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (ms < top_ms) { top_ms = ms; top = t; }
        }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    s->tuning = top;
    if (best) *best = top;
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    g_tune_cache.push_back({p->n_bands, p->n_bins, mixed, p->parts, logn, logt, top});
    return cudaGetLastError() == cudaSuccess ? VRC_OK : VRC_ERR_CUDA;
}
