// render.cu -- the renderer around the cache (Sec. 6): camera rays marched through the
// medium, cache look-ups at the march points, and adaptive record placement.
//
// Camera: pinhole at `pos` looking along `forward` (up = +z), vertical field of view
// `vfov_deg`, width x height pixels.  A pixel's ray enters the unit cube at s_in and is
// marched to s_end = min(first hit, cube exit) in `steps` equal segments; the march points
// are the segment midpoints (the paper's uniform ray marching, Sec. 6).  A pixel's value
// is sum_k ds sigma_s exp(-sigma_t (s_k - s_in)) L(x_k), L from Eq. radianceTaylor.
//
// Placement (Sec. 6: records are added where no valid record covers a point): candidates
// carry a level; wave `level` picks, in every cell of a 2^level grid over the cube, the
// uncovered candidate with the smallest index among those whose level is <= `level`.
// Full records are computed at the picked sites, the grid is rebuilt, the candidates are
// queried, and covered candidates leave the pool.
#include <algorithm>
#include <cmath>

#include "vrc_internal.cuh"

namespace {

struct Cam {
    float3 pos, fwd, right, up;
    float tan_half, aspect;
    int W, H;
};

__device__ __forceinline__ float3 norm3(float3 a) { return a * rsqrtf(dot3(a, a)); }

__device__ __forceinline__ float3 cam_dir(const Cam& c, int px, int py) {
    float x = (2.0f * ((float)px + 0.5f) / (float)c.W - 1.0f) * c.tan_half * c.aspect;
    float y = (1.0f - 2.0f * ((float)py + 0.5f) / (float)c.H) * c.tan_half;
    return norm3(c.fwd + c.right * x + c.up * y);
}

// [s_in, s_out] of the ray in the unit cube; false if it misses
__device__ __forceinline__ bool cube_span(float3 o, float3 d, float& s_in, float& s_out) {
    float t0 = -3.0e38f, t1 = 3.0e38f;
    const float oo[3] = {o.x, o.y, o.z}, dd[3] = {d.x, d.y, d.z};
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        if (dd[k] == 0.f) {
            if (oo[k] < 0.f || oo[k] > 1.f) return false;
            continue;
        }
        float a = (0.f - oo[k]) / dd[k], b = (1.f - oo[k]) / dd[k];
        t0 = fmaxf(t0, fminf(a, b));
        t1 = fminf(t1, fmaxf(a, b));
    }
    s_in = fmaxf(t0, 0.f);
    s_out = t1;
    return s_out > s_in;
}

// march span of pixel (px, py): entry, step and validity
__device__ __forceinline__ bool pixel_span(const DevScene& sc, const Cam& c, int px, int py, int steps, float3& o,
                                           float3& d, float& s_in, float& ds) {
    o = c.pos;
    d = cam_dir(c, px, py);
    float s_out;
    if (!cube_span(o, d, s_in, s_out)) return false;
    float3 e = o + d * s_in;
    float th;
    int prim = bvh_trace<false>(sc, e, d, VRC_TMIN, s_out - s_in + 1e-4f, &th);
    float len = prim >= 0 ? th : (s_out - s_in);
    if (!(len > 0.f)) return false;
    ds = len / (float)steps;
    return true;
}

__global__ void k_march_points(DevScene sc, Cam c, int x0, int y0, int w, int h, int stride, int steps, float* pts,
                               int* valid) {
    long long total = (long long)w * h * steps;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        int k = (int)(i % steps);
        long long pix = i / steps;
        int px = x0 + (int)(pix % w) * stride, py = y0 + (int)(pix / w) * stride;
        float3 o, d;
        float s_in, ds;
        bool ok = px < c.W && py < c.H && pixel_span(sc, c, px, py, steps, o, d, s_in, ds);
        float3 x = ok ? o + d * (s_in + ((float)k + 0.5f) * ds) : f3(0.f, 0.f, 0.f);
        pts[3 * i] = x.x;
        pts[3 * i + 1] = x.y;
        pts[3 * i + 2] = x.z;
        valid[i] = ok ? 1 : 0;
    }
}

__global__ void k_march_pixels(DevScene sc, Cam c, const int* pix, int n_pix, int steps, float* pts, int* valid) {
    long long total = (long long)n_pix * steps;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        int k = (int)(i % steps);
        int p = pix[i / steps];
        int px = p % c.W, py = p / c.W;
        float3 o, d;
        float s_in, ds;
        bool ok = pixel_span(sc, c, px, py, steps, o, d, s_in, ds);
        float3 x = ok ? o + d * (s_in + ((float)k + 0.5f) * ds) : f3(0.f, 0.f, 0.f);
        pts[3 * i] = x.x;
        pts[3 * i + 1] = x.y;
        pts[3 * i + 2] = x.z;
        valid[i] = ok ? 1 : 0;
    }
}

// Eq. radianceTaylor at x from the grid's compact records (order 1)
struct GridView {
    const float4* rec;
    const int* start;
    const int* list;
    int G;
    const float4* ell;   // ellipsoidal records' region matrices, NULL for spheres
};

__device__ __forceinline__ float3 cache_lookup(const GridView& g, float3 x, int& cnt) {
    int ix = min(g.G - 1, max(0, (int)floorf(x.x * g.G)));
    int iy = min(g.G - 1, max(0, (int)floorf(x.y * g.G)));
    int iz = min(g.G - 1, max(0, (int)floorf(x.z * g.G)));
    int cell = (ix * g.G + iy) * g.G + iz;
    int b = __ldg(&g.start[cell]), e = __ldg(&g.start[cell + 1]);
    float ar = 0.f, ag = 0.f, ab = 0.f, sw = 0.f;
    cnt = 0;
    for (int p = b; p < e; ++p) {
        int k = __ldg(&g.list[p]);
        float4 a = __ldg(&g.rec[4 * k]);
        float dx = x.x - a.x, dy = x.y - a.y, dz = x.z - a.z;
        float d2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
        if (!(d2 < a.w * a.w)) continue;
        float dd;
        if (g.ell) {   // ellipsoidal distance ratio sqrt(D^T M D)
            float4 m0 = __ldg(&g.ell[2 * k]), m1 = __ldg(&g.ell[2 * k + 1]);
            float r2e = fmaf(m0.x * dx, dx, fmaf(m0.w * dy, dy, m1.y * dz * dz)) +
                        2.0f * fmaf(m0.y * dx, dy, fmaf(m0.z * dx, dz, m1.x * dy * dz));
            if (!(r2e < 1.0f)) continue;
            dd = 1.0f - sqrtf(fmaxf(r2e, 0.f));
        } else {
            dd = 1.0f - sqrtf(d2) / a.w;
        }
        float4 r1 = __ldg(&g.rec[4 * k + 1]), r2 = __ldg(&g.rec[4 * k + 2]), r3 = __ldg(&g.rec[4 * k + 3]);
        float w = dd * dd * fmaf(-2.0f, dd, 3.0f);
        ar = fmaf(w, r1.x + fmaf(r1.w, dx, fmaf(r2.x, dy, r2.y * dz)), ar);
        ag = fmaf(w, r1.y + fmaf(r2.z, dx, fmaf(r2.w, dy, r3.x * dz)), ag);
        ab = fmaf(w, r1.z + fmaf(r3.y, dx, fmaf(r3.z, dy, r3.w * dz)), ab);
        sw += w;
        ++cnt;
    }
    float inv = cnt ? 1.0f / sw : 0.f;
    return f3(ar * inv, ag * inv, ab * inv);
}

// one thread per pixel: march, look up, accumulate; misses counted per pixel.  With a
// pixel list, thread i renders pixel pix[i] and writes at that pixel's index.  With a
// second grid (g2.rec != NULL) the radiance is the sum of both caches' look-ups and a
// march point counts as a miss once per cache that has no record for it.
__global__ void k_render(DevScene sc, Cam c, GridView g, GridView g2, int x0, int y0, int w, int h, int steps,
                         float* img, int* miss, const int* pix, int n_pix) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (pix ? n_pix : w * h)) return;
    int px, py;
    if (pix) {
        px = pix[i] % c.W;
        py = pix[i] / c.W;
        i = pix[i];
    } else {
        px = x0 + i % w;
        py = y0 + i / w;
    }
    float3 o, d, acc = f3(0.f, 0.f, 0.f);
    float s_in, ds;
    int nmiss = 0;
    if (px < c.W && py < c.H && pixel_span(sc, c, px, py, steps, o, d, s_in, ds)) {
        for (int k = 0; k < steps; ++k) {
            float s = ((float)k + 0.5f) * ds;
            float3 x = o + d * (s_in + s);
            int cnt;
            float3 L = cache_lookup(g, x, cnt);
            if (cnt == 0) ++nmiss;
            if (g2.rec) {
                L = L + cache_lookup(g2, x, cnt);
                if (cnt == 0) ++nmiss;
            }
            acc = acc + L * (ds * sc.sigma_s * __expf(-sc.sigma_t * s));
        }
    }
    img[3 * i] = acc.x;
    img[3 * i + 1] = acc.y;
    img[3 * i + 2] = acc.z;
    if (miss) miss[i] = nmiss;
}

// pixel values from per-point radiance (for the reference image: L at every march point)
__global__ void k_composite(DevScene sc, Cam c, int x0, int y0, int w, int h, int steps, const float* L, float* img) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= w * h) return;
    int px = x0 + i % w, py = y0 + i / w;
    float3 o, d, acc = f3(0.f, 0.f, 0.f);
    float s_in, ds;
    if (px < c.W && py < c.H && pixel_span(sc, c, px, py, steps, o, d, s_in, ds))
        for (int k = 0; k < steps; ++k) {
            float s = ((float)k + 0.5f) * ds;
            const float* l = L + 3 * ((size_t)i * steps + k);
            acc = acc + f3(l[0], l[1], l[2]) * (ds * sc.sigma_s * __expf(-sc.sigma_t * s));
        }
    img[3 * i] = acc.x;
    img[3 * i + 1] = acc.y;
    img[3 * i + 2] = acc.z;
}

// ---------------------------------------------------------------- placement
__global__ void k_site_claim(const float* pts, const int* level, int n, int lv, int G, int* cell_min, int* pool) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    int l = i < n ? level[i] : -1;
    // candidates still in the pool (any level), one atomic per warp
    const unsigned in_pool = __ballot_sync(0xffffffffu, l >= 0);
    if ((threadIdx.x & 31) == 0 && in_pool) atomicAdd(pool, __popc(in_pool));
    if (l < 0 || l > lv) return;
    int ix = min(G - 1, max(0, (int)floorf(pts[3 * i] * G)));
    int iy = min(G - 1, max(0, (int)floorf(pts[3 * i + 1] * G)));
    int iz = min(G - 1, max(0, (int)floorf(pts[3 * i + 2] * G)));
    atomicMin(&cell_min[((size_t)ix * G + iy) * G + iz], i);
}

__global__ void k_site_flag(const float* pts, const int* level, int n, int lv, int G, const int* cell_min, int* flag) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int l = level[i];
    int f = 0;
    if (l >= 0 && l <= lv) {
        int ix = min(G - 1, max(0, (int)floorf(pts[3 * i] * G)));
        int iy = min(G - 1, max(0, (int)floorf(pts[3 * i + 1] * G)));
        int iz = min(G - 1, max(0, (int)floorf(pts[3 * i + 2] * G)));
        f = cell_min[((size_t)ix * G + iy) * G + iz] == i ? 1 : 0;
    }
    flag[i] = f;
}

// block-local exclusive scan of flags, block totals to sums[blockIdx]
__global__ void k_flag_scan(const int* flag, int n, int* pos, int* sums) {
    __shared__ int s[1024];
    int i = blockIdx.x * 1024 + threadIdx.x;
    int v = i < n ? flag[i] : 0;
    s[threadIdx.x] = v;
    __syncthreads();
    for (int off = 1; off < 1024; off <<= 1) {
        int t = threadIdx.x >= off ? s[threadIdx.x - off] : 0;
        __syncthreads();
        s[threadIdx.x] += t;
        __syncthreads();
    }
    if (i < n) pos[i] = s[threadIdx.x] - v;
    if (threadIdx.x == 1023) sums[blockIdx.x] = s[1023];
}

__global__ void k_flag_tops(int* sums, int nblk, int* total) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        int run = 0;
        for (int b = 0; b < nblk; ++b) {
            int t = sums[b];
            sums[b] = run;
            run += t;
        }
        *total = run;
    }
}

__global__ void k_gather_sites(const float* pts, const int* flag, const int* pos, const int* sums, int n,
                               int* out_idx, float* out_pts) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n || !flag[i]) return;
    int j = pos[i] + sums[i / 1024];
    out_idx[j] = i;
    out_pts[3 * j] = pts[3 * i];
    out_pts[3 * j + 1] = pts[3 * i + 1];
    out_pts[3 * j + 2] = pts[3 * i + 2];
}

__global__ void k_nonzero(const int* v, int n, int* flag) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) flag[i] = v[i] != 0 ? 1 : 0;
}

__global__ void k_scatter_idx(const int* flag, const int* pos, const int* sums, int n, int* out) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n && flag[i]) out[pos[i] + sums[i / 1024]] = i;
}

__global__ void k_cover(const int* count, int n, int* level) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n && count[i] > 0) level[i] = -1;
}

// every pool candidate takes the level predicted for its cell's representative (the
// candidate with the smallest index in its cell of the 2^cell_level grid)
__global__ void k_rep_levels(const float* logr, const int* site_idx, int n_sites, float ratio, int lmin, int lmax,
                             int* rep_level) {
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n_sites) return;
    float R = __expf(logr[j]);
    int l = (int)ceilf(-log2f(fmaxf(ratio * R, 1e-6f)));
    rep_level[site_idx[j]] = min(lmax, max(lmin, l));
}
__global__ void k_cell_levels(const float* pts, int n, int G, const int* cell_min, const int* rep_level, int* level) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n || level[i] < 0) return;
    int ix = min(G - 1, max(0, (int)floorf(pts[3 * i] * G)));
    int iy = min(G - 1, max(0, (int)floorf(pts[3 * i + 1] * G)));
    int iz = min(G - 1, max(0, (int)floorf(pts[3 * i + 2] * G)));
    int rep = cell_min[((size_t)ix * G + iy) * G + iz];
    if (rep >= 0 && rep < n) level[i] = rep_level[rep];
}

// Sites of every level at once: a candidate of level l in [lmin, lmax] claims its cell of
// the 2^l grid; the cells of all levels share one array, level l's at offset
// (8^l - 8^lmin) / 7.
__device__ __forceinline__ long long ml_cell(const float* pts, int i, int l, int lmin) {
    const int G = 1 << l;
    const long long off = ((1ll << (3 * l)) - (1ll << (3 * lmin))) / 7;
    int ix = min(G - 1, max(0, (int)floorf(pts[3 * i] * G)));
    int iy = min(G - 1, max(0, (int)floorf(pts[3 * i + 1] * G)));
    int iz = min(G - 1, max(0, (int)floorf(pts[3 * i + 2] * G)));
    return off + ((long long)ix * G + iy) * G + iz;
}

__global__ void k_site_claim_ml(const float* pts, const int* level, int n, int lmin, int lmax, int* cell_min,
                                int* pool) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    int l = i < n ? level[i] : -1;
    const unsigned in_pool = __ballot_sync(0xffffffffu, l >= 0);
    if ((threadIdx.x & 31) == 0 && in_pool) atomicAdd(pool, __popc(in_pool));
    if (l < lmin || l > lmax) return;
    atomicMin(&cell_min[ml_cell(pts, i, l, lmin)], i);
}

__global__ void k_site_flag_ml(const float* pts, const int* level, int n, int lmin, int lmax, const int* cell_min,
                               int* flag) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int l = level[i];
    flag[i] = (l >= lmin && l <= lmax && cell_min[ml_cell(pts, i, l, lmin)] == i) ? 1 : 0;
}

__global__ void k_bump_levels(int* level, int n, int lmax) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n && level[i] >= 0) level[i] = min(level[i] + 1, lmax);
}

__global__ void k_retire_level(int* level, int n, int lv) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n && level[i] == lv) level[i] = -1;
}

// The learned radius (shifted by logr_offset: the predictor's log radius at its training
// tolerance plus (1/5) log of the ratio of tolerances, Eq. radiusAniso3D) is used only
// where the coarse ray set's own Hessian puts the error of a record of that radius within
// the tolerance: the error at R of Eq. radiusAniso3D, 4 pi |lambda| R^5 / (15 L), is at most
// eps exactly when R <= the coarse record's radius (same L, lambda and eps).  Elsewhere
// the prediction is replaced by logr_fallback (the candidate then starts with plain
// placement); their count goes to *n_fallback.  radius_coarse NULL: the shift only.
__global__ void k_mlp_fallback(const float* logr, float logr_offset, const float* radius_coarse, int n,
                               float logr_fallback, float* logr_out, int* n_fallback) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float l = logr[i] + logr_offset;
    bool ok = isfinite(l) && (!radius_coarse || __expf(l) <= radius_coarse[i]);
    logr_out[i] = ok ? l : logr_fallback;
    if (!ok) atomicAdd(n_fallback, 1);
}

__global__ void k_init_levels(const int* valid, int n, int start, int* level) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) level[i] = valid[i] ? start : -1;
}

// learned level of a candidate from its predicted log radius: the finest level whose
// cell is still at most `ratio` times the predicted radius, clamped to [lmin, lmax]
__global__ void k_levels_from_logr(const float* logr, int n, float ratio, int lmin, int lmax, int* level) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n || level[i] < 0) return;
    float R = __expf(logr[i]);
    int l = (int)ceilf(-log2f(fmaxf(ratio * R, 1e-6f)));
    level[i] = min(lmax, max(lmin, l));
}

Cam make_cam(const float* pos, const float* fwd, float vfov_deg, int W, int H) {
    Cam c;
    c.pos = make_float3(pos[0], pos[1], pos[2]);
    float fl = std::sqrt(fwd[0] * fwd[0] + fwd[1] * fwd[1] + fwd[2] * fwd[2]);
    c.fwd = make_float3(fwd[0] / fl, fwd[1] / fl, fwd[2] / fl);
    // right = fwd x (0,0,1), up = right x fwd
    float rx = c.fwd.y, ry = -c.fwd.x, rz = 0.f;
    float rl = std::sqrt(rx * rx + ry * ry);
    if (rl < 1e-6f) { rx = 1.f; ry = 0.f; rl = 1.f; }
    c.right = make_float3(rx / rl, ry / rl, rz);
    c.up = make_float3(c.right.y * c.fwd.z - c.right.z * c.fwd.y, c.right.z * c.fwd.x - c.right.x * c.fwd.z,
                       c.right.x * c.fwd.y - c.right.y * c.fwd.x);
    c.tan_half = std::tan(0.5f * vfov_deg * 3.14159265358979f / 180.f);
    c.aspect = (float)W / (float)H;
    c.W = W;
    c.H = H;
    return c;
}

}  // namespace

extern "C" int vrc_march_points(vrc_scene* s, const vrc_camera* cam, int32_t x0, int32_t y0, int32_t w, int32_t h,
                                int32_t stride, int32_t steps, float* d_pts, int32_t* d_valid, void* stream) {
    if (!s || !cam || w < 0 || h < 0 || stride < 1 || steps < 1 || !d_pts || !d_valid) return VRC_ERR_INVALID;
    if ((long long)w * h == 0) return VRC_OK;
    Cam c = make_cam(cam->pos, cam->forward, cam->vfov_deg, cam->width, cam->height);
    long long total = (long long)w * h * steps;
    int blocks = (int)std::min<long long>((total + 255) / 256, (long long)s->sm_count * 32);
    k_march_points<<<blocks, 256, 0, (cudaStream_t)stream>>>(s->dev, c, x0, y0, w, h, stride, steps, d_pts, d_valid);
    return cudaGetLastError() == cudaSuccess ? VRC_OK : VRC_ERR_CUDA;
}

static GridView grid_view(const vrc_grid* g) {
    if (!g) return GridView{nullptr, nullptr, nullptr, 1, nullptr};
    return GridView{g->rec, g->cell_start, g->cell_list, g->G, g->aniso ? g->ell : nullptr};
}

extern "C" int vrc_render(vrc_scene* s, const vrc_grid* grid, const vrc_grid* grid2, const vrc_camera* cam, int32_t x0,
                          int32_t y0, int32_t w, int32_t h, int32_t steps, float* d_img, int32_t* d_miss, void* stream) {
    if (!s || !grid || !cam || w < 0 || h < 0 || steps < 1 || !d_img) return VRC_ERR_INVALID;
    if ((long long)w * h == 0) return VRC_OK;
    Cam c = make_cam(cam->pos, cam->forward, cam->vfov_deg, cam->width, cam->height);
    if (grid->order != 1 || (grid2 && grid2->order != 1)) return VRC_ERR_INVALID;
    int n = w * h;
    k_render<<<(n + 127) / 128, 128, 0, (cudaStream_t)stream>>>(s->dev, c, grid_view(grid), grid_view(grid2), x0, y0,
                                                                  w, h, steps, d_img, d_miss, nullptr, 0);
    return cudaGetLastError() == cudaSuccess ? VRC_OK : VRC_ERR_CUDA;
}

extern "C" int vrc_composite(vrc_scene* s, const vrc_camera* cam, int32_t x0, int32_t y0, int32_t w, int32_t h,
                             int32_t steps, const float* d_L, float* d_img, void* stream) {
    if (!s || !cam || w < 0 || h < 0 || steps < 1 || !d_L || !d_img) return VRC_ERR_INVALID;
    if ((long long)w * h == 0) return VRC_OK;
    Cam c = make_cam(cam->pos, cam->forward, cam->vfov_deg, cam->width, cam->height);
    int n = w * h;
    k_composite<<<(n + 127) / 128, 128, 0, (cudaStream_t)stream>>>(s->dev, c, x0, y0, w, h, steps, d_L, d_img);
    return cudaGetLastError() == cudaSuccess ? VRC_OK : VRC_ERR_CUDA;
}

extern "C" int vrc_select_sites(const float* d_pts, const int32_t* d_level, int32_t n, int32_t level,
                                int32_t* d_scratch, int64_t scratch_ints, int32_t* d_site_idx, float* d_site_pts,
                                int32_t* h_count, int32_t* h_pool, void* stream) {
    if (!d_pts || !d_level || n < 0 || level < 0 || level > 8 || !d_scratch || !d_site_idx || !d_site_pts || !h_count)
        return VRC_ERR_INVALID;
    *h_count = 0;
    if (h_pool) *h_pool = 0;
    if (n == 0) return VRC_OK;
    const int G = 1 << level;
    const long long cells = (long long)G * G * G;
    const int nblk = (n + 1023) / 1024;
    if (scratch_ints < cells + 2LL * n + nblk + 2) return VRC_ERR_INVALID;
    cudaStream_t st = (cudaStream_t)stream;
    int* cell_min = d_scratch;
    int* flag = cell_min + cells;
    int* pos = flag + n;
    int* sums = pos + n;                  // [nblk] block sums, then the site count and the pool size
    VRC_CUDA_CHECK(cudaMemsetAsync(cell_min, 0x7f, sizeof(int) * cells, st));
    VRC_CUDA_CHECK(cudaMemsetAsync(sums + nblk + 1, 0, sizeof(int), st));
    int tb = 256, nb = (n + tb - 1) / tb;
    k_site_claim<<<nb, tb, 0, st>>>(d_pts, d_level, n, level, G, cell_min, sums + nblk + 1);
    k_site_flag<<<nb, tb, 0, st>>>(d_pts, d_level, n, level, G, cell_min, flag);
    k_flag_scan<<<nblk, 1024, 0, st>>>(flag, n, pos, sums);
    k_flag_tops<<<1, 32, 0, st>>>(sums, nblk, sums + nblk);
    k_gather_sites<<<nb, tb, 0, st>>>(d_pts, flag, pos, sums, n, d_site_idx, d_site_pts);
    int32_t both[2] = {0, 0};
    VRC_CUDA_CHECK(cudaMemcpyAsync(both, sums + nblk, 2 * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    VRC_CUDA_CHECK(cudaStreamSynchronize(st));
    *h_count = both[0];
    if (h_pool) *h_pool = both[1];
    return VRC_OK;
}

extern "C" int vrc_select_sites_levels(const float* d_pts, const int32_t* d_level, int32_t n, int32_t lmin,
                                       int32_t lmax, int32_t* d_scratch, int64_t scratch_ints, int32_t* d_site_idx,
                                       float* d_site_pts, int32_t* h_count, int32_t* h_pool, void* stream) {
    if (!d_pts || !d_level || n < 0 || lmin < 0 || lmax < lmin || lmax > 7 || !d_scratch || !d_site_idx ||
        !d_site_pts || !h_count)
        return VRC_ERR_INVALID;
    *h_count = 0;
    if (h_pool) *h_pool = 0;
    if (n == 0) return VRC_OK;
    const long long cells = ((1ll << (3 * (lmax + 1))) - (1ll << (3 * lmin))) / 7;
    const int nblk = (n + 1023) / 1024;
    if (scratch_ints < cells + 2LL * n + nblk + 2) return VRC_ERR_INVALID;
    cudaStream_t st = (cudaStream_t)stream;
    int* cell_min = d_scratch;
    int* flag = cell_min + cells;
    int* pos = flag + n;
    int* sums = pos + n;                  // [nblk] block sums, then the site count and the pool size
    VRC_CUDA_CHECK(cudaMemsetAsync(cell_min, 0x7f, sizeof(int) * cells, st));
    VRC_CUDA_CHECK(cudaMemsetAsync(sums + nblk + 1, 0, sizeof(int), st));
    int tb = 256, nb = (n + tb - 1) / tb;
    k_site_claim_ml<<<nb, tb, 0, st>>>(d_pts, d_level, n, lmin, lmax, cell_min, sums + nblk + 1);
    k_site_flag_ml<<<nb, tb, 0, st>>>(d_pts, d_level, n, lmin, lmax, cell_min, flag);
    k_flag_scan<<<nblk, 1024, 0, st>>>(flag, n, pos, sums);
    k_flag_tops<<<1, 32, 0, st>>>(sums, nblk, sums + nblk);
    k_gather_sites<<<nb, tb, 0, st>>>(d_pts, flag, pos, sums, n, d_site_idx, d_site_pts);
    int32_t both[2] = {0, 0};
    VRC_CUDA_CHECK(cudaMemcpyAsync(both, sums + nblk, 2 * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    VRC_CUDA_CHECK(cudaStreamSynchronize(st));
    *h_count = both[0];
    if (h_pool) *h_pool = both[1];
    return VRC_OK;
}

extern "C" int vrc_bump_levels(int32_t* d_level, int32_t n, int32_t lmax, void* stream) {
    if (n < 0 || (n > 0 && !d_level)) return VRC_ERR_INVALID;
    if (n == 0) return VRC_OK;
    k_bump_levels<<<(n + 255) / 256, 256, 0, (cudaStream_t)stream>>>(d_level, n, lmax);
    return cudaGetLastError() == cudaSuccess ? VRC_OK : VRC_ERR_CUDA;
}

extern "C" int vrc_update_coverage(const int32_t* d_count, int32_t n, int32_t* d_level, void* stream) {
    if (n < 0 || (n > 0 && (!d_count || !d_level))) return VRC_ERR_INVALID;
    if (n == 0) return VRC_OK;
    k_cover<<<(n + 255) / 256, 256, 0, (cudaStream_t)stream>>>(d_count, n, d_level);
    return cudaGetLastError() == cudaSuccess ? VRC_OK : VRC_ERR_CUDA;
}

extern "C" int vrc_retire_level(int32_t* d_level, int32_t n, int32_t level, void* stream) {
    if (n < 0 || (n > 0 && !d_level)) return VRC_ERR_INVALID;
    if (n == 0) return VRC_OK;
    k_retire_level<<<(n + 255) / 256, 256, 0, (cudaStream_t)stream>>>(d_level, n, level);
    return cudaGetLastError() == cudaSuccess ? VRC_OK : VRC_ERR_CUDA;
}

extern "C" int vrc_mlp_fallback(const float* d_logr, int32_t n, float logr_offset, const float* d_radius_coarse,
                                float logr_fallback, float* d_logr_out, int32_t* d_n_fallback, void* stream) {
    if (n < 0 || (n > 0 && (!d_logr || !d_logr_out || !d_n_fallback))) return VRC_ERR_INVALID;
    if (n == 0) return VRC_OK;
    k_mlp_fallback<<<(n + 255) / 256, 256, 0, (cudaStream_t)stream>>>(d_logr, logr_offset, d_radius_coarse, n,
                                                                    logr_fallback, d_logr_out, d_n_fallback);
    return cudaGetLastError() == cudaSuccess ? VRC_OK : VRC_ERR_CUDA;
}

extern "C" int vrc_levels_from_radius(const float* d_logr, int32_t n, float cell_over_radius, int32_t lmin,
                                      int32_t lmax, int32_t* d_level, void* stream) {
    if (n < 0 || lmin < 0 || lmax < lmin || lmax > 8 || !(cell_over_radius > 0.f)) return VRC_ERR_INVALID;
    if (n == 0) return VRC_OK;
    if (!d_logr || !d_level) return VRC_ERR_INVALID;
    k_levels_from_logr<<<(n + 255) / 256, 256, 0, (cudaStream_t)stream>>>(d_logr, n, cell_over_radius, lmin, lmax,
                                                                          d_level);
    return cudaGetLastError() == cudaSuccess ? VRC_OK : VRC_ERR_CUDA;
}

extern "C" int vrc_init_levels(const int32_t* d_valid, int32_t n, int32_t start_level, int32_t* d_level, void* stream) {
    if (n < 0 || start_level < 0 || (n > 0 && (!d_valid || !d_level))) return VRC_ERR_INVALID;
    if (n == 0) return VRC_OK;
    k_init_levels<<<(n + 255) / 256, 256, 0, (cudaStream_t)stream>>>(d_valid, n, start_level, d_level);
    return cudaGetLastError() == cudaSuccess ? VRC_OK : VRC_ERR_CUDA;
}

extern "C" int vrc_levels_by_cell(const float* d_pts, int32_t n, int32_t cell_level, const int32_t* d_scratch,
                                  const int32_t* d_site_idx, const float* d_site_logr, int32_t n_sites,
                                  float cell_over_radius, int32_t lmin, int32_t lmax, int32_t* d_rep_level,
                                  int32_t* d_level, void* stream) {
    if (n < 0 || n_sites < 0 || cell_level < 0 || cell_level > 8 || lmin < 0 || lmax < lmin || lmax > 8 ||
        !(cell_over_radius > 0.f))
        return VRC_ERR_INVALID;
    if (n == 0 || n_sites == 0) return VRC_OK;
    if (!d_pts || !d_scratch || !d_site_idx || !d_site_logr || !d_rep_level || !d_level) return VRC_ERR_INVALID;
    cudaStream_t st = (cudaStream_t)stream;
    k_rep_levels<<<(n_sites + 255) / 256, 256, 0, st>>>(d_site_logr, d_site_idx, n_sites, cell_over_radius, lmin, lmax,
                                                        d_rep_level);
    k_cell_levels<<<(n + 255) / 256, 256, 0, st>>>(d_pts, n, 1 << cell_level, d_scratch, d_rep_level, d_level);
    return cudaGetLastError() == cudaSuccess ? VRC_OK : VRC_ERR_CUDA;
}

extern "C" int vrc_march_pixels(vrc_scene* s, const vrc_camera* cam, const int32_t* d_pix, int32_t n_pix, int32_t steps,
                                float* d_pts, int32_t* d_valid, void* stream) {
    if (!s || !cam || n_pix < 0 || steps < 1) return VRC_ERR_INVALID;
    if (n_pix == 0) return VRC_OK;
    if (!d_pix || !d_pts || !d_valid) return VRC_ERR_INVALID;
    Cam c = make_cam(cam->pos, cam->forward, cam->vfov_deg, cam->width, cam->height);
    long long total = (long long)n_pix * steps;
    int blocks = (int)std::min<long long>((total + 255) / 256, (long long)s->sm_count * 32);
    k_march_pixels<<<blocks, 256, 0, (cudaStream_t)stream>>>(s->dev, c, d_pix, n_pix, steps, d_pts, d_valid);
    return cudaGetLastError() == cudaSuccess ? VRC_OK : VRC_ERR_CUDA;
}

extern "C" int vrc_render_pixels(vrc_scene* s, const vrc_grid* grid, const vrc_grid* grid2, const vrc_camera* cam,
                                 const int32_t* d_pix, int32_t n_pix, int32_t steps, float* d_img, int32_t* d_miss,
                                 void* stream) {
    if (!s || !grid || !cam || n_pix < 0 || steps < 1 || grid->order != 1) return VRC_ERR_INVALID;
    if (grid2 && grid2->order != 1) return VRC_ERR_INVALID;
    if (n_pix == 0) return VRC_OK;
    if (!d_pix || !d_img) return VRC_ERR_INVALID;
    Cam c = make_cam(cam->pos, cam->forward, cam->vfov_deg, cam->width, cam->height);
    k_render<<<(n_pix + 127) / 128, 128, 0, (cudaStream_t)stream>>>(s->dev, c, grid_view(grid), grid_view(grid2), 0, 0,
                                                                      0, 0, steps, d_img, d_miss, d_pix, n_pix);
    return cudaGetLastError() == cudaSuccess ? VRC_OK : VRC_ERR_CUDA;
}

extern "C" int vrc_compact_indices(const int32_t* d_flags, int32_t n, int32_t* d_scratch, int64_t scratch_ints,
                                   int32_t* d_idx, int32_t* h_count, void* stream) {
    if (n < 0 || !h_count) return VRC_ERR_INVALID;
    *h_count = 0;
    if (n == 0) return VRC_OK;
    const int nblk = (n + 1023) / 1024;
    if (!d_flags || !d_scratch || !d_idx || scratch_ints < 2LL * n + nblk + 1) return VRC_ERR_INVALID;
    cudaStream_t st = (cudaStream_t)stream;
    int* flag = d_scratch;
    int* pos = flag + n;
    int* sums = pos + n;
    k_nonzero<<<(n + 255) / 256, 256, 0, st>>>(d_flags, n, flag);
    k_flag_scan<<<nblk, 1024, 0, st>>>(flag, n, pos, sums);
    k_flag_tops<<<1, 32, 0, st>>>(sums, nblk, sums + nblk);
    k_scatter_idx<<<(n + 255) / 256, 256, 0, st>>>(flag, pos, sums, n, d_idx);
    VRC_CUDA_CHECK(cudaMemcpyAsync(h_count, sums + nblk, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    VRC_CUDA_CHECK(cudaStreamSynchronize(st));
    return VRC_OK;
}
