// flat.cu -- records of the paper's two-dimensional world (Sec. 3; Sec. 4 in 2D; App. A;
// App. B; Eq. radiusAniso2D).
//
// The intrinsic planar model: light travels, scatters and is absorbed in the plane,
// radiance from a point source falls off as 1/r, the (isotropic) phase function is
// 1/(2 pi) over the circle.  Geometry is a set of line segments in the unit square.
// A record at x traces N equal-angle strata (one jittered ray each), marches the
// rays into distance shells, and sums over every shell's cells -- the segments between
// angularly adjacent vertices -- the radiance L_j = f T L_o theta_j with its gradient
// and Hessian (product rule; T from App. A at the cell's furthest endpoint, theta_j
// the angle the cell subtends, App. B).  The angle's derivatives are taken here from
// theta = atan2(A, B), A = (y0 - x) x (y1 - x), B = (y0 - x) . (y1 - x):
//   grad A = ((y0 - y1).y, (y1 - y0).x) (constant), grad B = -(y0 - x) - (y1 - x),
//   H B = 2 I, grad theta = (B grad A - A grad B) / D, D = A^2 + B^2,
//   H theta = sym[(grad A grad B^T - grad B grad A^T - 2 A I) / D
//                 - (B grad A - A grad B)(2 A grad A + 2 B grad B)^T / D^2],
// which equal App. B's arccos expressions (signed) wherever those are defined.
//
// Outputs go to the 3D record layout in the plane z = 0.5 (zero z components), so the
// 3D record grid and query kernels serve 2D records unchanged.
//
// One block per record at a time (persistent blocks, atomic work counter); the ray
// set, the shell's vertex radiance and the per-thread sums live in shared memory and
// registers; segments are read through L1 (2D scenes are a few KB).
#include <cmath>
#include <vector>

#include "vrc_internal.cuh"

struct vrc2d_scene {
    float4* d_seg;       // [n] (x0, y0, x1, y1)
    float4* d_prim;      // [n][2] (unit normal x, y, -, -), (albedo rgb, -)
    int n_segs;
    int n_lights;
    float2 lpos[VRC_MAX_LIGHTS];
    float3 lI[VRC_MAX_LIGHTS];
    float sigma_s, sigma_t;
    int sm_count;
    int* d_counter;
};

namespace {

constexpr int NT2 = 128;
constexpr float PLANE_Z = 0.5f;
constexpr float TMIN2 = 1e-6f;

struct Scene2View {
    const float4* __restrict__ seg;
    const float4* __restrict__ prim;
    int n_segs, n_lights;
    float2 lpos[VRC_MAX_LIGHTS];
    float3 lI[VRC_MAX_LIGHTS];
    float sigma_s, sigma_t;
};

struct Rec2Args {
    const float* pos;    // [n][2]
    int n, N;
    float dt, eps, r_min, r_max;
    uint64_t seed;
    long long rec_base;
    int parts;
    vrc_records_view out;
    int* counter;
};

__device__ __forceinline__ float cross2(float2 a, float2 b) { return a.x * b.y - a.y * b.x; }

// ray x + t d against segment a + u (b - a); u widened by 2e-7 so rays through a shared
// endpoint cannot slip between two segments
__device__ __forceinline__ bool seg_hit(float2 x, float2 d, float4 s, float& t) {
    float2 e = make_float2(s.z - s.x, s.w - s.y), w = make_float2(s.x - x.x, s.y - x.y);
    float den = cross2(d, e);
    if (den == 0.f) return false;
    float inv = 1.0f / den;
    float tt = cross2(w, e) * inv;
    float u = cross2(w, d) * inv;
    if (!(tt > TMIN2) || u < -2e-7f || u > 1.0f + 2e-7f) return false;
    t = tt;
    return true;
}

__device__ int closest_seg(const Scene2View& sc, float2 x, float2 d, float& t_out) {
    int best = -1;
    float bt = 3.0e38f;
    for (int i = 0; i < sc.n_segs; ++i) {
        float t;
        if (seg_hit(x, d, __ldg(&sc.seg[i]), t) && t < bt) { bt = t; best = i; }
    }
    t_out = bt;
    return best;
}

__device__ bool occluded_seg(const Scene2View& sc, float2 o, float2 d, float limit) {
    for (int i = 0; i < sc.n_segs; ++i) {
        float t;
        if (seg_hit(o, d, __ldg(&sc.seg[i]), t) && t < limit) return true;
    }
    return false;
}

__device__ __forceinline__ float square_exit(float2 x, float2 d) {
    float t = 3.0e38f;
    if (d.x > 0.f) t = fminf(t, (1.f - x.x) / d.x); else if (d.x < 0.f) t = fminf(t, -x.x / d.x);
    if (d.y > 0.f) t = fminf(t, (1.f - x.y) / d.y); else if (d.y < 0.f) t = fminf(t, -x.y / d.y);
    return t;
}

// radiance toward x of a surface point (two-sided Lambertian curve, f_r = albedo / 2)
// or of a medium point (isotropic single scattering, f = 1 / (2 pi)); 1/d falloff
__device__ float3 vertex_radiance2(const Scene2View& sc, float2 y, int prim, float2 d_in) {
    float3 Lo = make_float3(0.f, 0.f, 0.f);
    float2 n = make_float2(0.f, 0.f);
    float3 alb = make_float3(0.f, 0.f, 0.f);
    float2 o = y;
    if (prim >= 0) {
        float4 p0 = __ldg(&sc.prim[2 * prim]), p1 = __ldg(&sc.prim[2 * prim + 1]);
        n = make_float2(p0.x, p0.y);
        if (n.x * d_in.x + n.y * d_in.y > 0.f) n = make_float2(-n.x, -n.y);   // face x
        alb = make_float3(0.5f * p1.x, 0.5f * p1.y, 0.5f * p1.z);
        o = make_float2(y.x + 1e-5f * n.x, y.y + 1e-5f * n.y);
    }
    for (int l = 0; l < sc.n_lights; ++l) {
        float2 tl = make_float2(sc.lpos[l].x - o.x, sc.lpos[l].y - o.y);
        float dist = sqrtf(tl.x * tl.x + tl.y * tl.y);
        float2 ld = make_float2(tl.x / dist, tl.y / dist);
        float cs = 1.f;
        if (prim >= 0) {
            cs = n.x * ld.x + n.y * ld.y;
            if (cs <= 0.f) continue;
        }
        if (occluded_seg(sc, o, ld, dist)) continue;
        float k = cs * __expf(-sc.sigma_t * dist) / dist;
        if (prim >= 0) {
            Lo.x += alb.x * sc.lI[l].x * k;
            Lo.y += alb.y * sc.lI[l].y * k;
            Lo.z += alb.z * sc.lI[l].z * k;
        } else {
            const float f = 1.0f / (2.0f * VRC_PI_F);
            Lo.x += f * sc.lI[l].x * k;
            Lo.y += f * sc.lI[l].y * k;
            Lo.z += f * sc.lI[l].z * k;
        }
    }
    return Lo;
}

__device__ __forceinline__ void neu(float& s, float& c, float x) {
    float t = s + x;
    if (fabsf(s) >= fabsf(x)) c += (s - t) + x;
    else c += (x - t) + s;
    s = t;
}

// 18 sums per part: per channel L, grad (2), hess (xx, xy, yy)
struct Acc2 {
    float s[18], c[18];
};

// One cell (y0, y1) of a shell: angle and derivatives (atan2 form), T at the furthest
// endpoint(s) (App. A; mean over exact ties), product rule, weight w.  Returns false for
// a degenerate cell (A = B = 0).
__device__ bool cell2(float2 x, float2 y0, float2 y1, float t0, float t1, float3 L0, float3 L1, float sigma_t, float w,
                      Acc2& acc) {
    float2 u = make_float2(y0.x - x.x, y0.y - x.y), v = make_float2(y1.x - x.x, y1.y - x.y);
    float A = cross2(u, v), B = u.x * v.x + u.y * v.y;
    float D = A * A + B * B;
    if (!(D > 0.f)) return false;
    float th = atan2f(A, B);
    float2 gA = make_float2(u.y - v.y, v.x - u.x), gB = make_float2(-(u.x + v.x), -(u.y + v.y));
    float iD = 1.0f / D;
    float2 N = make_float2(B * gA.x - A * gB.x, B * gA.y - A * gB.y);
    float2 gth = make_float2(N.x * iD, N.y * iD);
    float2 gD = make_float2(2.f * (A * gA.x + B * gB.x), 2.f * (A * gA.y + B * gB.y));
    // symmetric part: the grad A grad B^T - grad B grad A^T term is antisymmetric and
    // drops out; divide by D twice in turn (D^2 alone can leave the float range)
    float hxx = (-2.f * A - N.x * gD.x * iD) * iD;
    float hyy = (-2.f * A - N.y * gD.y * iD) * iD;
    float hxy = (-0.5f * (N.x * gD.y + N.y * gD.x) * iD) * iD;
    // furthest endpoint(s)
    float tm = fmaxf(t0, t1);
    bool f0 = t0 == tm, f1 = t1 == tm;
    float nf = (f0 && f1) ? 0.5f : 1.0f;
    float Lr[3] = {0.f, 0.f, 0.f}, gr[3][2] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}},
          hr[3][3] = {{0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}};
#pragma unroll
    for (int q = 0; q < 2; ++q) {
        if (!(q == 0 ? f0 : f1)) continue;
        float2 y = q == 0 ? y0 : y1;
        float3 Lo = q == 0 ? L0 : L1;
        float wx = x.x - y.x, wy = x.y - y.y;
        float r = sqrtf(wx * wx + wy * wy);
        float ir = 1.0f / r;
        float T = __expf(-sigma_t * r);
        float gx = -sigma_t * wx * ir * T, gy = -sigma_t * wy * ir * T;
        float a = (sigma_t * sigma_t * ir * ir + sigma_t * ir * ir * ir) * T, b = -sigma_t * ir * T;
        float Hxx = a * wx * wx + b, Hxy = a * wx * wy, Hyy = a * wy * wy + b;
        float lo[3] = {Lo.x * nf, Lo.y * nf, Lo.z * nf};
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            Lr[c] += lo[c] * T;
            gr[c][0] += lo[c] * gx;
            gr[c][1] += lo[c] * gy;
            hr[c][0] += lo[c] * Hxx;
            hr[c][1] += lo[c] * Hxy;
            hr[c][2] += lo[c] * Hyy;
        }
    }
    const float wf = w * (1.0f / (2.0f * VRC_PI_F));
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        neu(acc.s[6 * c + 0], acc.c[6 * c + 0], wf * Lr[c] * th);
        neu(acc.s[6 * c + 1], acc.c[6 * c + 1], wf * (gr[c][0] * th + Lr[c] * gth.x));
        neu(acc.s[6 * c + 2], acc.c[6 * c + 2], wf * (gr[c][1] * th + Lr[c] * gth.y));
        neu(acc.s[6 * c + 3], acc.c[6 * c + 3], wf * (hr[c][0] * th + 2.f * gr[c][0] * gth.x + Lr[c] * hxx));
        neu(acc.s[6 * c + 4], acc.c[6 * c + 4],
            wf * (hr[c][1] * th + gr[c][0] * gth.y + gr[c][1] * gth.x + Lr[c] * hxy));
        neu(acc.s[6 * c + 5], acc.c[6 * c + 5], wf * (hr[c][2] * th + 2.f * gr[c][1] * gth.y + Lr[c] * hyy));
    }
    return true;
}

// shared memory: ray (dx, dy, t_end, -) [N], vertex radiance rgb [3][N], per-thread sums
// [NT][42] (surface-shell cell sums 18, medium-shell cell sums 18, MC surface 3, MC
// medium 3), their block totals [42], misc ints
constexpr int NCOL = 42;
size_t rec2_smem(int N) { return (size_t)N * 16 + (size_t)N * 12 + (size_t)NT2 * NCOL * 4 + NCOL * 4 + 8 * 4; }

// Six blocks per SM (registers capped at 80, a few bytes spilled): 24 warps hide the
// fixed-latency chains of the segment tests and cell arithmetic better than the 16 warps of
// four blocks at 110 registers (measured on the 2D mid workload: 2.26 -> 1.82 ms per 4,096
// records; five blocks, 96 registers: 1.93 ms; a larger shared-memory carveout: no change).
__global__ void __launch_bounds__(NT2, 6) k_records2d(Scene2View sc, Rec2Args a) {
    extern __shared__ float4 sm4[];
    const int N = a.N;
    float4* ray = sm4;
    float* Lr = reinterpret_cast<float*>(ray + N);
    float* Lg = Lr + N;
    float* Lb = Lg + N;
    float* red = Lb + N;                 // [NT][NCOL]
    float* tot = red + NT2 * NCOL;       // [NCOL]
    int* misc = reinterpret_cast<int*>(tot + NCOL);
    __shared__ int s_rec;
    const int tid = threadIdx.x;
    const float f = 1.0f / (2.0f * VRC_PI_F);
    const float wmc = 2.0f * VRC_PI_F / (float)N;
    float* mine = red + tid * NCOL;
    for (;;) {
        if (tid == 0) {
            int item = atomicAdd(a.counter, 1);
            s_rec = item < a.n ? item : a.n;
            misc[0] = 0;
            misc[1] = 0;
            misc[2] = 0;
            misc[3] = 0;
        }
        __syncthreads();
        const int rec = s_rec;
        if (rec >= a.n) break;
        const long long rid = a.rec_base + rec;
        const float2 x = make_float2(a.pos[2 * rec], a.pos[2 * rec + 1]);
        float ms[3] = {0.f, 0.f, 0.f}, msc[3] = {0.f, 0.f, 0.f};   // MC sums, surface
        float mm[3] = {0.f, 0.f, 0.f}, mmc[3] = {0.f, 0.f, 0.f};   // MC sums, medium
        float tmax = 0.f;
        // ---------------- primary rays (surface shell vertices)
        for (int j = tid; j < N; j += NT2) {
            double ang = ((double)j + (double)jitter_dev(a.seed, rid, 0, j, 2)) / (double)N;
            double sd, cd;
            sincospi(2.0 * ang, &sd, &cd);
            float2 d = make_float2((float)cd, (float)sd);
            float t;
            int prim = closest_seg(sc, x, d, t);
            float3 Lo = make_float3(0.f, 0.f, 0.f);
            if (prim >= 0) {
                if (a.parts != 2) Lo = vertex_radiance2(sc, make_float2(x.x + d.x * t, x.y + d.y * t), prim, d);
                float w = wmc * f * __expf(-sc.sigma_t * t);
                neu(ms[0], msc[0], w * Lo.x);
                neu(ms[1], msc[1], w * Lo.y);
                neu(ms[2], msc[2], w * Lo.z);
            } else {
                t = square_exit(x, d);
            }
            if (a.out.hit_prim) {                    // debug: the primary hit decisions
                a.out.hit_prim[(size_t)rec * a.out.dbg_stride + j] = prim;
                a.out.hit_t[(size_t)rec * a.out.dbg_stride + j] = t;
            }
            ray[j] = make_float4(d.x, d.y, t, 0.f);
            Lr[j] = Lo.x;
            Lg[j] = Lo.y;
            Lb[j] = Lo.z;
            tmax = fmaxf(tmax, t);
        }
        atomicMax(&misc[0], __float_as_int(tmax));   // non-negative floats order as ints
        __syncthreads();
        const int K = a.parts == 1 ? 0 : (int)ceilf(__int_as_float(misc[0]) / a.dt);
        const float wms = sc.sigma_s * a.dt;
        Acc2 acc;
        for (int e = 0; e < 18; ++e) acc.s[e] = acc.c[e] = 0.f;
        int cells = 0, fars = 0, degen = 0;
        for (int k = 0; k <= K; ++k) {
            const float tk = ((float)k - 0.5f) * a.dt;
            if (k == 1) {
                // the surface shell is done: park its sums, start the medium shells
                for (int e = 0; e < 18; ++e) {
                    mine[e] = acc.s[e] + acc.c[e];
                    acc.s[e] = acc.c[e] = 0.f;
                }
            }
            if (k >= 1) {
                __syncthreads();                 // the previous shell's cells are done
                for (int j = tid; j < N; j += NT2) {
                    float4 rv = ray[j];
                    float3 Lo = make_float3(0.f, 0.f, 0.f);
                    if (tk < rv.z) {
                        Lo = vertex_radiance2(sc, make_float2(x.x + rv.x * tk, x.y + rv.y * tk), -1,
                                              make_float2(0.f, 0.f));
                        float w = wms * wmc * f * __expf(-sc.sigma_t * tk);
                        neu(mm[0], mmc[0], w * Lo.x);
                        neu(mm[1], mmc[1], w * Lo.y);
                        neu(mm[2], mmc[2], w * Lo.z);
                    }
                    Lr[j] = Lo.x;
                    Lg[j] = Lo.y;
                    Lb[j] = Lo.z;
                }
                __syncthreads();
            }
            if (a.parts == 2 && k == 0) continue;        // multiple-scattering cache: no surface shell
            const float w = k == 0 ? 1.0f : wms;
            for (int j = tid; j < N; j += NT2) {
                int j1 = j + 1 == N ? 0 : j + 1;
                float4 r0 = ray[j], r1 = ray[j1];
                float t0 = (k == 0 || !(tk < r0.z)) ? r0.z : tk;
                float t1 = (k == 0 || !(tk < r1.z)) ? r1.z : tk;
                float3 L0 = make_float3(Lr[j], Lg[j], Lb[j]), L1 = make_float3(Lr[j1], Lg[j1], Lb[j1]);
                float tm = fmaxf(t0, t1);
                bool lit = (t0 == tm && (L0.x != 0.f || L0.y != 0.f || L0.z != 0.f)) ||
                           (t1 == tm && (L1.x != 0.f || L1.y != 0.f || L1.z != 0.f));
                if (!lit) continue;
                float2 y0 = make_float2(x.x + r0.x * t0, x.y + r0.y * t0);
                float2 y1 = make_float2(x.x + r1.x * t1, x.y + r1.y * t1);
                if (cell2(x, y0, y1, t0, t1, L0, L1, sc.sigma_t, w, acc)) {
                    ++cells;
                    fars += (t0 == t1) ? 2 : 1;
                } else {
                    ++degen;
                }
            }
        }
        // ---------------- deterministic block reduction (fixed thread order)
        for (int e = 0; e < 18; ++e) {
            float v = acc.s[e] + acc.c[e];
            if (K == 0) {
                mine[e] = v;
                mine[18 + e] = 0.f;
            } else {
                mine[18 + e] = v;
            }
        }
        for (int c = 0; c < 3; ++c) {
            mine[36 + c] = ms[c] + msc[c];
            mine[39 + c] = mm[c] + mmc[c];
        }
        atomicAdd(&misc[1], cells);
        atomicAdd(&misc[2], degen);
        atomicAdd(&misc[3], fars);
        __syncthreads();
        if (tid < NCOL) {
            float sum = 0.f, cmp = 0.f;
            for (int t = 0; t < NT2; ++t) neu(sum, cmp, red[t * NCOL + tid]);
            tot[tid] = sum + cmp;
        }
        __syncthreads();
        // ---------------- outputs (3D layout, plane z = 0.5)
        const vrc_records_view& o = a.out;
        if (tid < 3) {
            int c = tid;
            float ls = tot[36 + c], lm = tot[39 + c];
            o.L[3 * rec + c] = ls + lm;
            if (o.L_ss) o.L_ss[3 * rec + c] = ls;
            if (o.L_ms) o.L_ms[3 * rec + c] = lm;
            o.pos[3 * rec + c] = c == 0 ? x.x : (c == 1 ? x.y : PLANE_Z);
        } else if (tid >= 32 && tid < 35) {
            int c = tid - 32;
            const float* ps = tot + 6 * c;          // surface shell
            const float* pm = tot + 18 + 6 * c;     // medium shells
            float gs[3] = {ps[1], ps[2], 0.f}, gm[3] = {pm[1], pm[2], 0.f};
            float hs[6] = {ps[3], ps[4], 0.f, ps[5], 0.f, 0.f}, hm[6] = {pm[3], pm[4], 0.f, pm[5], 0.f, 0.f};
            for (int e = 0; e < 3; ++e) {
                o.grad[9 * rec + 3 * c + e] = gs[e] + gm[e];
                if (o.grad_ss) o.grad_ss[9 * rec + 3 * c + e] = gs[e];
                if (o.grad_ms) o.grad_ms[9 * rec + 3 * c + e] = gm[e];
            }
            for (int e = 0; e < 6; ++e) {
                o.hess[18 * rec + 6 * c + e] = hs[e] + hm[e];
                if (o.hess_ss) o.hess_ss[18 * rec + 6 * c + e] = hs[e];
                if (o.hess_ms) o.hess_ms[18 * rec + 6 * c + e] = hm[e];
            }
            if (o.L_ff) o.L_ff[3 * rec + c] = ps[0] + pm[0];
        } else if (tid == 64) {
            bool finite = true;
            for (int e = 0; e < NCOL; ++e)
                if (!isfinite(tot[e])) finite = false;
            int st = finite ? 0 : VRC_REC_NONFINITE;
            if (misc[2] > 0) st |= VRC_REC_DEGENERATE;
            o.status[rec] = st;
            if (o.n_cells) o.n_cells[rec] = misc[1];
            if (o.n_far) o.n_far[rec] = misc[3];
            if (o.n_shells) o.n_shells[rec] = K;
        }
        __syncthreads();
    }
}

// Radius stage in 2D (Eq. radiusAniso2D): R = (4 L_Y eps / (pi max|lambda|))^(1/4) from the
// 2x2 luminance Hessian; the ellipse's principal radii per eigenvalue, embedded with the
// normal axis (eigenvalue 0: r_max).
__global__ void k_radius2d(Rec2Args a) {
    int rec = blockIdx.x * blockDim.x + threadIdx.x;
    if (rec >= a.n) return;
    const vrc_records_view& o = a.out;
    const double Y[3] = {0.2126, 0.7152, 0.0722};
    const float* H = o.hess + 18 * (size_t)rec;
    double hxx = 0, hxy = 0, hyy = 0, LY = 0;
    for (int c = 0; c < 3; ++c) {
        hxx += Y[c] * (double)H[6 * c + 0];
        hxy += Y[c] * (double)H[6 * c + 1];
        hyy += Y[c] * (double)H[6 * c + 3];
        LY += Y[c] * (double)o.L[3 * rec + c];
    }
    double m = 0.5 * (hxx + hyy), dl = sqrt(0.25 * (hxx - hyy) * (hxx - hyy) + hxy * hxy);
    double l0 = m - dl, l1 = m + dl;
    double lmax = fmax(fabs(l0), fabs(l1));
    int st = o.status[rec];
    bool bad = (st & VRC_REC_NONFINITE) || !isfinite(LY) || !isfinite(lmax);
    double R;
    const double PI = 3.14159265358979323846;
    if (bad) { st |= VRC_REC_NONFINITE | VRC_REC_CLAMP_LO; R = a.r_min; }
    else if (!(LY > 0.0)) { st |= VRC_REC_CLAMP_LO; R = a.r_min; }
    else if (lmax == 0.0) { st |= VRC_REC_CLAMP_HI; R = a.r_max; }
    else {
        R = pow(4.0 * LY * (double)a.eps / (PI * lmax), 0.25);
        if (R < a.r_min) { st |= VRC_REC_CLAMP_LO; R = a.r_min; }
        if (R > a.r_max) { st |= VRC_REC_CLAMP_HI; R = a.r_max; }
    }
    o.radius[rec] = (float)R;
    if (o.log_radius) o.log_radius[rec] = (float)log(R);
    o.status[rec] = st;
    // embedded eigenvalues (l0, l1, 0) ascending, with their axes
    double lam[3] = {l0, l1, 0.0};
    double ax[3][3];
    // eigenvector of l1 in the plane: angle t = atan2(2 hxy, hxx - hyy) / 2
    double t = 0.5 * atan2(2.0 * hxy, hxx - hyy);
    double c1 = cos(t), s1 = sin(t);
    double v1[3] = {c1, s1, 0.0}, v0[3] = {-s1, c1, 0.0}, vz[3] = {0.0, 0.0, 1.0};
    int idx[3] = {0, 1, 2};
    const double* vec[3] = {v0, v1, vz};
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 2 - i; ++j)
            if (lam[idx[j]] > lam[idx[j + 1]]) { int tt = idx[j]; idx[j] = idx[j + 1]; idx[j + 1] = tt; }
    for (int i = 0; i < 3; ++i)
        for (int k = 0; k < 3; ++k) ax[i][k] = vec[idx[i]][k];
    if (o.eig)
        for (int i = 0; i < 3; ++i) o.eig[3 * rec + i] = (float)lam[idx[i]];
    for (int i = 0; i < 3; ++i) {
        double al = fabs(lam[idx[i]]), Ri;
        if (bad || !(LY > 0.0)) Ri = a.r_min;
        else if (al == 0.0) Ri = a.r_max;
        else Ri = fmin((double)a.r_max, fmax((double)a.r_min, pow(4.0 * LY * (double)a.eps / (PI * al), 0.25)));
        if (o.radii) o.radii[3 * rec + i] = (float)Ri;
        if (o.axes)
            for (int k = 0; k < 3; ++k) o.axes[9 * rec + 3 * i + k] = (float)ax[i][k];
    }
}

}  // namespace

extern "C" int vrc2d_build_scene(const float* segs, int32_t n_segs, const float* albedo, float sigma_s, float sigma_a,
                                 const vrc2d_point_light* lights, int32_t n_lights, vrc2d_scene** out) {
    if (!out || n_segs < 0 || (n_segs > 0 && (!segs || !albedo)) || n_lights < 0 || n_lights > VRC_MAX_LIGHTS ||
        (n_lights > 0 && !lights) || !(sigma_s >= 0.f) || !(sigma_a >= 0.f))
        return VRC_ERR_INVALID;
    *out = nullptr;
    std::vector<float4> seg((size_t)n_segs > 0 ? n_segs : 1), prim(2 * ((size_t)n_segs > 0 ? n_segs : 1));
    for (int i = 0; i < n_segs; ++i) {
        const float* s = segs + 4 * i;
        float ex = s[2] - s[0], ey = s[3] - s[1];
        float len = std::sqrt(ex * ex + ey * ey);
        if (!(len > 0.f) || !std::isfinite(len)) return VRC_ERR_INVALID;
        seg[i] = make_float4(s[0], s[1], s[2], s[3]);
        prim[2 * i] = make_float4(-ey / len, ex / len, 0.f, 0.f);
        prim[2 * i + 1] = make_float4(albedo[3 * i], albedo[3 * i + 1], albedo[3 * i + 2], 0.f);
    }
    vrc2d_scene* s = new vrc2d_scene();
    s->n_segs = n_segs;
    s->n_lights = n_lights;
    for (int l = 0; l < n_lights; ++l) {
        s->lpos[l] = make_float2(lights[l].pos[0], lights[l].pos[1]);
        s->lI[l] = make_float3(lights[l].intensity[0], lights[l].intensity[1], lights[l].intensity[2]);
    }
    s->sigma_s = sigma_s;
    s->sigma_t = sigma_s + sigma_a;
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&s->sm_count, cudaDevAttrMultiProcessorCount, dev);
    if (cudaMalloc((void**)&s->d_seg, sizeof(float4) * seg.size()) != cudaSuccess ||
        cudaMalloc((void**)&s->d_prim, sizeof(float4) * prim.size()) != cudaSuccess ||
        cudaMalloc((void**)&s->d_counter, sizeof(int)) != cudaSuccess) {
        vrc2d_destroy_scene(s);
        return VRC_ERR_OOM;
    }
    if (cudaMemcpy(s->d_seg, seg.data(), sizeof(float4) * seg.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(s->d_prim, prim.data(), sizeof(float4) * prim.size(), cudaMemcpyHostToDevice) != cudaSuccess) {
        vrc2d_destroy_scene(s);
        return VRC_ERR_CUDA;
    }
    *out = s;
    return VRC_OK;
}

extern "C" void vrc2d_destroy_scene(vrc2d_scene* s) {
    if (!s) return;
    cudaFree(s->d_seg);
    cudaFree(s->d_prim);
    cudaFree(s->d_counter);
    delete s;
}

extern "C" int vrc2d_compute_records(vrc2d_scene* s, const float* d_pos, int32_t n, const vrc_record_params* p,
                                     const vrc_records_view* out, void* stream) {
    if (!s || !p || !out || n < 0) return VRC_ERR_INVALID;
    if (n == 0) return VRC_OK;
    if (!d_pos || !out->L || !out->grad || !out->hess || !out->radius || !out->status || !out->pos)
        return VRC_ERR_INVALID;
    const int N = p->n_bins;
    if (p->n_bands != 1 || N < 3 || !(p->dt > 0.f) || !(p->eps > 0.f) || !(p->r_min > 0.f) ||
        !(p->r_max >= p->r_min) || p->parts < 0 || p->parts > 2)
        return VRC_ERR_INVALID;
    if (N > 4096) return VRC_ERR_UNSUPPORTED;
    if (out->hit_prim && (!out->hit_t || out->dbg_stride < N)) return VRC_ERR_INVALID;
    size_t smem = rec2_smem(N);
    cudaStream_t st = (cudaStream_t)stream;
    Scene2View sv;
    sv.seg = s->d_seg;
    sv.prim = s->d_prim;
    sv.n_segs = s->n_segs;
    sv.n_lights = s->n_lights;
    for (int l = 0; l < VRC_MAX_LIGHTS; ++l) {
        sv.lpos[l] = s->lpos[l];
        sv.lI[l] = s->lI[l];
    }
    sv.sigma_s = s->sigma_s;
    sv.sigma_t = s->sigma_t;
    Rec2Args a;
    a.pos = d_pos;
    a.n = n;
    a.N = N;
    a.dt = p->dt;
    a.eps = p->eps;
    a.r_min = p->r_min;
    a.r_max = p->r_max;
    a.seed = p->seed;
    a.rec_base = p->rec_base;
    a.parts = p->parts;
    a.out = *out;
    a.counter = s->d_counter;
    if (cudaFuncSetAttribute(k_records2d, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return VRC_ERR_UNSUPPORTED;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_records2d, NT2, smem) != cudaSuccess || per_sm < 1)
        return VRC_ERR_UNSUPPORTED;
    int grid = per_sm * s->sm_count;
    if (grid > n) grid = n;
    VRC_CUDA_CHECK(cudaMemsetAsync(s->d_counter, 0, sizeof(int), st));
    k_records2d<<<grid, NT2, smem, st>>>(sv, a);
    k_radius2d<<<(n + 127) / 128, 128, 0, st>>>(a);
    return cudaGetLastError() == cudaSuccess ? VRC_OK : VRC_ERR_CUDA;
}
