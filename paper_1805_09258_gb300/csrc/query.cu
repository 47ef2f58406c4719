// query.cu -- radiance interpolation from cache records (Eq. radianceTaylor, Sec. 5).
//
// L(x') = sum_{k in C} w_k [L_k + grad L_k . (x' - x_k) (+ 1/2 D^T H_k D)] / sum_k w_k,
// C = {k : |x' - x_k| < R_k}, w = 3 d^2 - 2 d^3, d = 1 - |x' - x_k| / R_k.
//
// The paper looks records up in an octree (Sec. 6); here the lookup is a uniform grid
// over the unit cube whose cells list (CSR) every record whose sphere overlaps the
// cell, so a query reads exactly one list.  Queries are first binned by cell (count,
// scan, scatter) so the threads of a warp share one list: its record rows are read as
// warp-wide broadcasts from L1.  Every buffer is owned by the vrc_grid object.
//
// Ellipsoidal records (Eq. radiusAniso3D per eigenvalue): the distance ratio |D| / R_k
// becomes rho = sqrt(D^T M_k D) with M_k = sum_i v_i v_i^T / R_i^2; a record is listed in
// the cells that meet both its bounding box and its bounding sphere.
#include <algorithm>
#include <cmath>
#include <vector>

#include "vrc_internal.cuh"

namespace {

constexpr int SCAN_BLOCK = 1024;

__global__ void k_pack(const vrc_records_view v, int n, int order, float4* rec, float4* hess) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const float* p = v.pos + 3 * k;
    const float* L = v.L + 3 * k;
    const float* g = v.grad + 9 * k;
    rec[4 * k] = make_float4(p[0], p[1], p[2], v.radius ? v.radius[k] : 0.f);
    rec[4 * k + 1] = make_float4(L[0], L[1], L[2], g[0]);
    rec[4 * k + 2] = make_float4(g[1], g[2], g[3], g[4]);
    rec[4 * k + 3] = make_float4(g[5], g[6], g[7], g[8]);
    if (order == 2) {
        const float* h = v.hess + 18 * k;
        for (int e = 0; e < 5; ++e)
            hess[5 * k + e] = make_float4(h[4 * e], h[4 * e + 1], 4 * e + 2 < 18 ? h[4 * e + 2] : 0.f,
                                          4 * e + 3 < 18 ? h[4 * e + 3] : 0.f);
    }
}

// ellipsoidal records: M = sum_i v_i v_i^T / R_i^2, bounding-box half extents
// e_j = sqrt(sum_i R_i^2 v_ij^2), largest radius in rec .w
__global__ void k_pack_ellipsoid(const vrc_records_view v, int n, float4* rec, float4* ell, float4* ext) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const float* r = v.radii + 3 * k;
    const float* ax = v.axes + 9 * k;
    float m[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f}, e2[3] = {0.f, 0.f, 0.f};
    float rmax = 0.f;
    for (int i = 0; i < 3; ++i) {
        const float* u = ax + 3 * i;
        float inv = 1.0f / (r[i] * r[i]);
        m[0] = fmaf(u[0] * u[0], inv, m[0]);
        m[1] = fmaf(u[0] * u[1], inv, m[1]);
        m[2] = fmaf(u[0] * u[2], inv, m[2]);
        m[3] = fmaf(u[1] * u[1], inv, m[3]);
        m[4] = fmaf(u[1] * u[2], inv, m[4]);
        m[5] = fmaf(u[2] * u[2], inv, m[5]);
        for (int j = 0; j < 3; ++j) e2[j] = fmaf(r[i] * r[i], u[j] * u[j], e2[j]);
        rmax = fmaxf(rmax, r[i]);
    }
    rec[4 * k].w = rmax;
    ell[2 * k] = make_float4(m[0], m[1], m[2], m[3]);
    ell[2 * k + 1] = make_float4(m[4], m[5], 0.f, 0.f);
    // the box may not exceed the bounding sphere (float rounding of the axes)
    ext[k] = make_float4(fminf(sqrtf(e2[0]), rmax), fminf(sqrtf(e2[1]), rmax), fminf(sqrtf(e2[2]), rmax), rmax);
}

__device__ __forceinline__ bool sphere_meets_cell(float3 c, float R, int ix, int iy, int iz, float h) {
    float lx = ix * h, ly = iy * h, lz = iz * h;
    float dx = fmaxf(fmaxf(lx - c.x, c.x - (lx + h)), 0.f);
    float dy = fmaxf(fmaxf(ly - c.y, c.y - (ly + h)), 0.f);
    float dz = fmaxf(fmaxf(lz - c.z, c.z - (lz + h)), 0.f);
    return dx * dx + dy * dy + dz * dz < R * R;
}

// count (fill = false) or fill (fill = true) the cells each record's sphere overlaps;
// with `ext` (ellipsoidal records) only the cells within its bounding box.  One warp per
// record, its lanes over the cells of the record's box: a record meets hundreds of cells,
// and the lanes' atomics are then in flight together.
template <bool FILL>
__global__ void k_insert(const float4* rec, const float4* ext, int n, int G, int* counts, const int* start,
                         int* list) {
    int k = (int)(((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    int lane = threadIdx.x & 31;
    if (k >= n) return;
    float4 a = rec[4 * k];
    float3 c = make_float3(a.x, a.y, a.z);
    float R = a.w;
    float ex = R, ey = R, ez = R;
    if (ext) {
        float4 e = ext[k];
        ex = e.x, ey = e.y, ez = e.z;
    }
    float h = 1.0f / G;
    int x0 = max(0, (int)floorf((c.x - ex) * G)), x1 = min(G - 1, (int)floorf((c.x + ex) * G));
    int y0 = max(0, (int)floorf((c.y - ey) * G)), y1 = min(G - 1, (int)floorf((c.y + ey) * G));
    int z0 = max(0, (int)floorf((c.z - ez) * G)), z1 = min(G - 1, (int)floorf((c.z + ez) * G));
    int ny = y1 - y0 + 1, nz = z1 - z0 + 1;
    int total = (x1 - x0 + 1) * ny * nz;
    for (int t = lane; t < total; t += 32) {
        int ix = x0 + t / (ny * nz), r = t % (ny * nz);
        int iy = y0 + r / nz, iz = z0 + r % nz;
        if (!sphere_meets_cell(c, R, ix, iy, iz, h)) continue;
        int cell = (ix * G + iy) * G + iz;
        int slot = atomicAdd(&counts[cell], 1);
        if (FILL) list[start[cell] + slot] = k;
    }
}

// Sort each cell's list ascending (a deterministic summation order for the queries).
// Record ids in a list are distinct, so each element's position is the number of smaller
// elements (a rank sort).  Grids of up to WARP_SORT_CELLS cells: one block per cell
// (k_sort_cells).  Finer grids (small radii, placement's fine waves at 64^3 cells): one warp
// per cell, up to 64 entries two per lane in registers, ranked by shuffles, up to WSORT_CAP
// in the warp's shared buffer, longer lists handed to k_sort_lists (a block per list); a
// block per cell there spent its time on launching blocks for lists of a few tens
// (measured rebuilds: 3,725 records of radius 0.02-0.1, 0.36 -> 0.28 ms; on the benchmark's
// grid, 4,096 records, the block per cell stays 10 us faster).
constexpr int WARP_SORT_CELLS = 1 << 17;
constexpr int WSORT_CAP = 512;
__global__ void __launch_bounds__(256) k_sort_lists_warp(const int* start, int ncell, int* list, int* long_cells,
                                                         int* n_long) {
    __shared__ int buf[8][WSORT_CAP];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int cell = blockIdx.x * 8 + w; cell < ncell; cell += gridDim.x * 8) {
        const int b = start[cell], e = start[cell + 1], len = e - b;
        if (len <= 1) continue;
        if (len <= 64) {
            const int v0 = lane < len ? list[b + lane] : 0x7fffffff;
            const int v1 = lane + 32 < len ? list[b + 32 + lane] : 0x7fffffff;
            int r0 = 0, r1 = 0;
#pragma unroll 8
            for (int j = 0; j < 32; ++j) {
                const int u0 = __shfl_sync(0xffffffffu, v0, j), u1 = __shfl_sync(0xffffffffu, v1, j);
                r0 += (u0 < v0 ? 1 : 0) + (u1 < v0 ? 1 : 0);
                r1 += (u0 < v1 ? 1 : 0) + (u1 < v1 ? 1 : 0);
            }
            if (lane < len) list[b + r0] = v0;
            if (lane + 32 < len) list[b + r1] = v1;
        } else if (len <= WSORT_CAP) {
            for (int i = lane; i < len; i += 32) buf[w][i] = list[b + i];
            __syncwarp();
            for (int i = lane; i < len; i += 32) {
                const int v = buf[w][i];
                int r = 0;
                for (int j = 0; j < len; ++j) r += buf[w][j] < v ? 1 : 0;
                list[b + r] = v;
            }
            __syncwarp();
        } else if (lane == 0) {
            long_cells[atomicAdd(n_long, 1)] = cell;
        }
    }
}

constexpr int SORT_CAP = 4096;

// one block per cell: rank sort in shared memory; lists longer than its buffer: an
// insertion sort by one thread
__global__ void __launch_bounds__(256) k_sort_cells(const int* start, int ncell, int* list) {
    __shared__ int buf[SORT_CAP];
    int cell = blockIdx.x;
    if (cell >= ncell) return;
    int b = start[cell], e = start[cell + 1], len = e - b;
    if (len <= 1) return;
    if (len > SORT_CAP) {
        if (threadIdx.x == 0)
            for (int i = b + 1; i < e; ++i) {
                int v = list[i], j = i - 1;
                while (j >= b && list[j] > v) { list[j + 1] = list[j]; --j; }
                list[j + 1] = v;
            }
        return;
    }
    for (int i = threadIdx.x; i < len; i += blockDim.x) buf[i] = list[b + i];
    __syncthreads();
    for (int i = threadIdx.x; i < len; i += blockDim.x) {
        int v = buf[i], r = 0;
        for (int j = 0; j < len; ++j) r += buf[j] < v;
        list[b + r] = v;
    }
}

// the lists longer than WSORT_CAP of a fine grid, one block each (as k_sort_cells)
__global__ void __launch_bounds__(256) k_sort_lists(const int* start, const int* long_cells, const int* n_long,
                                                    int* list) {
    __shared__ int buf[SORT_CAP];
    for (int li = blockIdx.x; li < *n_long; li += gridDim.x) {
        const int cell = long_cells[li];
        int b = start[cell], e = start[cell + 1], len = e - b;
        if (len > SORT_CAP) {
            if (threadIdx.x == 0)
                for (int i = b + 1; i < e; ++i) {
                    int v = list[i], j = i - 1;
                    while (j >= b && list[j] > v) { list[j + 1] = list[j]; --j; }
                    list[j + 1] = v;
                }
            __syncthreads();
            continue;
        }
        for (int i = threadIdx.x; i < len; i += blockDim.x) buf[i] = list[b + i];
        __syncthreads();
        for (int i = threadIdx.x; i < len; i += blockDim.x) {
            int v = buf[i], r = 0;
            for (int j = 0; j < len; ++j) r += buf[j] < v;
            list[b + r] = v;
        }
        __syncthreads();
    }
}

// exclusive scan of in[0, m) into out[0, m]; out[m] = total.  Two-level, block sums in tmp.
__global__ void k_scan_blocks(const int* in, int m, int* out, int* tmp) {
    __shared__ int s[SCAN_BLOCK];
    int i = blockIdx.x * SCAN_BLOCK + threadIdx.x;
    int v = i < m ? in[i] : 0;
    s[threadIdx.x] = v;
    __syncthreads();
    for (int off = 1; off < SCAN_BLOCK; off <<= 1) {
        int t = threadIdx.x >= off ? s[threadIdx.x - off] : 0;
        __syncthreads();
        s[threadIdx.x] += t;
        __syncthreads();
    }
    if (i < m) out[i] = s[threadIdx.x] - v;
    if (threadIdx.x == SCAN_BLOCK - 1) tmp[blockIdx.x] = s[threadIdx.x];
}

__global__ void k_scan_tops(int* tmp, int nblk) {
    // one thread: block counts are few (<= a few hundred)
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        int run = 0;
        for (int b = 0; b < nblk; ++b) {
            int t = tmp[b];
            tmp[b] = run;
            run += t;
        }
        tmp[nblk] = run;
    }
}

__global__ void k_scan_add(int* out, int m, const int* tmp, int nblk) {
    int i = blockIdx.x * SCAN_BLOCK + threadIdx.x;
    if (i < m) out[i] += tmp[blockIdx.x];
    if (i == 0) out[m] = tmp[nblk];
}

int exclusive_scan(const int* in, int m, int* out, int* tmp, cudaStream_t st) {
    int nblk = (m + SCAN_BLOCK - 1) / SCAN_BLOCK;
    k_scan_blocks<<<nblk, SCAN_BLOCK, 0, st>>>(in, m, out, tmp);
    k_scan_tops<<<1, 32, 0, st>>>(tmp, nblk);
    k_scan_add<<<nblk, SCAN_BLOCK, 0, st>>>(out, m, tmp, nblk);
    return cudaGetLastError() == cudaSuccess ? VRC_OK : VRC_ERR_CUDA;
}

__device__ __forceinline__ int cell_of(float3 q, int G) {
    int ix = min(G - 1, max(0, (int)floorf(q.x * G)));
    int iy = min(G - 1, max(0, (int)floorf(q.y * G)));
    int iz = min(G - 1, max(0, (int)floorf(q.z * G)));
    return (ix * G + iy) * G + iz;
}

__global__ void k_bin_queries(const float* q, int nq, int G, int* qcell, int* qrank, int* counts) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nq) return;
    int c = cell_of(make_float3(q[3 * i], q[3 * i + 1], q[3 * i + 2]), G);
    qcell[i] = c;
    qrank[i] = atomicAdd(&counts[c], 1);
}

// each query's point and index at its place in cell order (the query kernel then reads
// them coalesced, without a dependent gather)
__global__ void k_scatter_queries(const float* q, const int* qcell, const int* qrank, const int* start, int nq,
                                  float4* pts) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nq) return;
    pts[start[qcell[i]] + qrank[i]] = make_float4(q[3 * i], q[3 * i + 1], q[3 * i + 2], __int_as_float(i));
}

// one thread per query, in cell order
template <int ORDER, bool ANISO>
__global__ void __launch_bounds__(256) k_query(const float4* __restrict__ rec, const float4* __restrict__ hess,
                                               const float4* __restrict__ ell,
                                               const int* __restrict__ cell_start, const int* __restrict__ list,
                                               int G, const float4* __restrict__ pts, int nq,
                                               float* __restrict__ rgb, int* __restrict__ status) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31;
    const bool active = s < nq;
    const unsigned am = __ballot_sync(0xffffffffu, active);
    if (am == 0u) return;                                // the whole warp is past the queries
    int i = 0, c = 0;
    float3 x = make_float3(0.f, 0.f, 0.f);
    if (active) {
        const float4 p = pts[s];
        i = __float_as_int(p.w);
        x = make_float3(p.x, p.y, p.z);
        c = cell_of(x, G);
    }
    // the warp's queries are binned by cell: when they all fall in one cell, its record rows
    // are staged in shared memory 32 at a time by the lanes together, and every lane reads
    // them from there (the same rows, in the same order, as the per-lane loop below)
    const int c0 = __shfl_sync(0xffffffffu, c, __ffs(am) - 1);
    const bool uniform = __all_sync(0xffffffffu, !active || c == c0);
    const int b = cell_start[uniform ? c0 : c], e = cell_start[(uniform ? c0 : c) + 1];
    float ar = 0.f, ag = 0.f, ab = 0.f, sw = 0.f;
    int cnt = 0;
    // candidate record k with row `row` (its first float4 already in a)
    auto candidate = [&](int k, float4 a, const float4* row, bool staged) {
        float dx = x.x - a.x, dy = x.y - a.y, dz = x.z - a.z;
        float d2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
        if (!(d2 < a.w * a.w)) return;
        float dd;
        if (ANISO) {
            float4 m0 = __ldg(&ell[2 * k]), m1 = __ldg(&ell[2 * k + 1]);
            float r2e = fmaf(m0.x * dx, dx, fmaf(m0.w * dy, dy, m1.y * dz * dz)) +
                        2.0f * fmaf(m0.y * dx, dy, fmaf(m0.z * dx, dz, m1.x * dy * dz));
            if (!(r2e < 1.0f)) return;
            dd = 1.0f - sqrtf(fmaxf(r2e, 0.f));
        } else {
            dd = 1.0f - sqrtf(d2) / a.w;
        }
        const float4 r1 = staged ? row[1] : __ldg(row + 1), r2 = staged ? row[2] : __ldg(row + 2),
                     r3 = staged ? row[3] : __ldg(row + 3);
        float w = dd * dd * fmaf(-2.0f, dd, 3.0f);
        float vr = r1.x + fmaf(r1.w, dx, fmaf(r2.x, dy, r2.y * dz));
        float vg = r1.y + fmaf(r2.z, dx, fmaf(r2.w, dy, r3.x * dz));
        float vb = r1.z + fmaf(r3.y, dx, fmaf(r3.z, dy, r3.w * dz));
        if (ORDER == 2) {
            float4 h0 = __ldg(&hess[5 * k]), h1 = __ldg(&hess[5 * k + 1]), h2 = __ldg(&hess[5 * k + 2]),
                   h3 = __ldg(&hess[5 * k + 3]), h4 = __ldg(&hess[5 * k + 4]);
            float hh[18] = {h0.x, h0.y, h0.z, h0.w, h1.x, h1.y, h1.z, h1.w, h2.x,
                            h2.y, h2.z, h2.w, h3.x, h3.y, h3.z, h3.w, h4.x, h4.y};
            float qv[3];
#pragma unroll
            for (int ch = 0; ch < 3; ++ch) {
                const float* H = hh + 6 * ch;
                qv[ch] = 0.5f * (H[0] * dx * dx + H[3] * dy * dy + H[5] * dz * dz) +
                         (H[1] * dx * dy + H[2] * dx * dz + H[4] * dy * dz);
            }
            vr += qv[0];
            vg += qv[1];
            vb += qv[2];
        }
        ar = fmaf(w, vr, ar);
        ag = fmaf(w, vg, ag);
        ab = fmaf(w, vb, ab);
        sw += w;
        ++cnt;
    };
    if (uniform) {
        __shared__ float4 rows[256 / 32][32][4];
        __shared__ int ids[256 / 32][32];
        float4(*rw)[4] = rows[threadIdx.x >> 5];
        int* kw = ids[threadIdx.x >> 5];
        for (int p0 = b; p0 < e; p0 += 32) {
            const int n = min(32, e - p0);
            if (lane < n) {
                const int k = __ldg(&list[p0 + lane]);
                kw[lane] = k;
#pragma unroll
                for (int h = 0; h < 4; ++h) rw[lane][h] = __ldg(&rec[4 * k + h]);
            }
            __syncwarp();
            if (active)
                for (int j = 0; j < n; ++j) candidate(kw[j], rw[j][0], rw[j], true);
            __syncwarp();
        }
    } else if (active) {
        for (int p = b; p < e; ++p) {
            const int k = __ldg(&list[p]);
            candidate(k, __ldg(&rec[4 * k]), rec + 4 * k, false);
        }
    }
    if (!active) return;
    float inv = cnt ? 1.0f / sw : 0.0f;
    rgb[3 * i] = ar * inv;
    rgb[3 * i + 1] = ag * inv;
    rgb[3 * i + 2] = ab * inv;
    status[i] = cnt;
}

template <typename T>
int dev_alloc(T** p, size_t count) {
    if (cudaMalloc((void**)p, std::max<size_t>(count, 1) * sizeof(T)) != cudaSuccess) {
        *p = nullptr;
        return VRC_ERR_OOM;
    }
    return VRC_OK;
}

}  // namespace

extern "C" void vrc_destroy_grid(vrc_grid* g) {
    if (!g) return;
    cudaFree(g->rec);
    cudaFree(g->hess);
    cudaFree(g->ell);
    cudaFree(g->ext);
    cudaFree(g->cell_start);
    cudaFree(g->cell_list);
    cudaFree(g->q_cell);
    cudaFree(g->q_rank);
    cudaFree(g->q_pts);
    cudaFree(g->q_count);
    cudaFree(g->scan_tmp);
    delete g;
}

namespace {

// grow a buffer of `cap` elements to at least `need` (its contents are not kept)
template <typename T>
int grow(T** p, long long* cap, long long need) {
    if (need < 1) need = 1;
    if (*cap >= need) return VRC_OK;
    cudaFree(*p);
    *p = nullptr;
    *cap = 0;
    if (cudaMalloc((void**)p, sizeof(T) * (size_t)need) != cudaSuccess) {
        *p = nullptr;
        return VRC_ERR_OOM;
    }
    *cap = need;
    return VRC_OK;
}

// (re)build grid g from n records, reusing its buffers where they are large enough
int fill_grid(vrc_grid* g, const vrc_records_view* v, int32_t n, int32_t order, bool aniso, cudaStream_t st) {
    if (!v || n < 0 || (order != 1 && order != 2)) return VRC_ERR_INVALID;
    if (n > 0 && (!v->pos || !v->L || !v->grad || (order == 2 && !v->hess))) return VRC_ERR_INVALID;
    if (n > 0 && (aniso ? (!v->radii || !v->axes) : !v->radius)) return VRC_ERR_INVALID;
    // cell size: about a quarter of the median radius (ellipsoids: of the geometric mean
    // of the principal radii), at most 64 cells per axis
    int G = 1;
    if (n > 0) {
        std::vector<float> R(aniso ? 3 * (size_t)n : (size_t)n);
        if (cudaMemcpyAsync(R.data(), aniso ? v->radii : v->radius, sizeof(float) * R.size(), cudaMemcpyDeviceToHost,
                            st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess)
            return VRC_ERR_CUDA;
        if (aniso) {
            for (int k = 0; k < n; ++k) R[k] = std::cbrt(R[3 * k] * R[3 * k + 1] * R[3 * k + 2]);
            R.resize(n);
        }
        std::nth_element(R.begin(), R.begin() + n / 2, R.end());
        float med = R[n / 2];
        if (!(med > 0.f) || !std::isfinite(med)) med = 0.1f;
        G = (int)std::ceil(4.0f / med);
        G = std::max(1, std::min(64, G));
    }
    const int ncell = G * G * G;
    const int nblk = (ncell + 1 + SCAN_BLOCK - 1) / SCAN_BLOCK;
    long long ext_cap = g->ell_cap / 2;   // ext holds one float4 per record, ell two
    int rc = VRC_OK;
    if ((rc = grow(&g->rec, &g->rec_cap, 4 * (long long)n)) ||
        (order == 2 && (rc = grow(&g->hess, &g->hess_cap, 5 * (long long)n))) ||
        (rc = grow(&g->cell_start, &g->cell_cap, (long long)ncell + 1)) ||
        (rc = grow(&g->scan_tmp, &g->scan_cap, (long long)nblk + 1)))
        return rc;
    if (aniso) {
        if (g->ell_cap < 2 * (long long)n) {
            cudaFree(g->ext);
            g->ext = nullptr;
            ext_cap = 0;
            if ((rc = grow(&g->ell, &g->ell_cap, 2 * (long long)n)) || (rc = grow(&g->ext, &ext_cap, (long long)n)))
                return rc;
        }
    }
    // query scratch: cell counts sized like cell_start
    if (g->q_count == nullptr || g->cell_cap > g->q_count_cap) {
        cudaFree(g->q_count);
        g->q_count = nullptr;
        g->q_count_cap = 0;
        if (cudaMalloc((void**)&g->q_count, sizeof(int) * (size_t)g->cell_cap) != cudaSuccess) return VRC_ERR_OOM;
        g->q_count_cap = g->cell_cap;
    }
    g->n = n;
    g->order = order;
    g->aniso = aniso ? 1 : 0;
    g->G = G;
    if (n > 0) {
        int tb = 256, nbk = (n + tb - 1) / tb;
        k_pack<<<nbk, tb, 0, st>>>(*v, n, order, g->rec, g->hess);
        if (aniso) k_pack_ellipsoid<<<nbk, tb, 0, st>>>(*v, n, g->rec, g->ell, g->ext);
        cudaMemsetAsync(g->q_count, 0, sizeof(int) * (ncell + 1), st);
        int nwb = (int)(((long long)n * 32 + tb - 1) / tb);   // one warp per record
        k_insert<false><<<nwb, tb, 0, st>>>(g->rec, aniso ? g->ext : nullptr, n, G, g->q_count, nullptr, nullptr);
        exclusive_scan(g->q_count, ncell, g->cell_start, g->scan_tmp, st);
        int total = 0;
        if (cudaMemcpyAsync(&total, g->cell_start + ncell, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess)
            return VRC_ERR_CUDA;
        g->entries = total;
        if ((rc = grow(&g->cell_list, &g->list_cap, (long long)total))) return rc;
        cudaMemsetAsync(g->q_count, 0, sizeof(int) * (ncell + 1), st);
        k_insert<true><<<nwb, tb, 0, st>>>(g->rec, aniso ? g->ext : nullptr, n, G, g->q_count, g->cell_start,
                                           g->cell_list);
        if (ncell <= WARP_SORT_CELLS) {
            k_sort_cells<<<ncell, 256, 0, st>>>(g->cell_start, ncell, g->cell_list);
        } else {
            // the fill cursors (q_count) are free again: long lists' cells and their count
            int* long_cells = g->q_count;
            int* n_long = g->q_count + ncell;
            cudaMemsetAsync(n_long, 0, sizeof(int), st);
            int sm = 0, dev = 0;
            cudaGetDevice(&dev);
            cudaDeviceGetAttribute(&sm, cudaDevAttrMultiProcessorCount, dev);
            sm = std::max(sm, 1);
            const int wblk = std::max(1, std::min((ncell + 7) / 8, 8 * sm));
            k_sort_lists_warp<<<wblk, 256, 0, st>>>(g->cell_start, ncell, g->cell_list, long_cells, n_long);
            k_sort_lists<<<std::max(1, std::min(ncell, 16 * sm)), 256, 0, st>>>(g->cell_start, long_cells, n_long,
                                                                                 g->cell_list);
        }
    } else {
        g->entries = 0;
        cudaMemsetAsync(g->cell_start, 0, sizeof(int) * (ncell + 1), st);
        if ((rc = grow(&g->cell_list, &g->list_cap, 1))) return rc;
    }
    return cudaGetLastError() == cudaSuccess ? VRC_OK : VRC_ERR_CUDA;
}

int build_grid(const vrc_records_view* v, int32_t n, int32_t order, bool aniso, vrc_grid** out, void* stream) {
    if (!out) return VRC_ERR_INVALID;
    *out = nullptr;
    vrc_grid* g = new vrc_grid();
    int rc = fill_grid(g, v, n, order, aniso, (cudaStream_t)stream);
    if (rc != VRC_OK) {
        vrc_destroy_grid(g);
        return rc;
    }
    *out = g;
    return VRC_OK;
}

}  // namespace

extern "C" int vrc_build_record_grid(const vrc_records_view* v, int32_t n, int32_t order, vrc_grid** out,
                                     void* stream) {
    return build_grid(v, n, order, false, out, stream);
}

extern "C" int vrc_build_record_grid_aniso(const vrc_records_view* v, int32_t n, int32_t order, vrc_grid** out,
                                           void* stream) {
    return build_grid(v, n, order, true, out, stream);
}

extern "C" int vrc_rebuild_record_grid(vrc_grid* g, const vrc_records_view* v, int32_t n, int32_t order, int32_t aniso,
                                       void* stream) {
    if (!g || aniso < 0 || aniso > 1) return VRC_ERR_INVALID;
    return fill_grid(g, v, n, order, aniso != 0, (cudaStream_t)stream);
}

extern "C" int vrc_query_inscatter(const vrc_grid* gc, const float* d_q, int32_t nq, float* d_rgb,
                                   int32_t* d_status, void* stream) {
    if (!gc || nq < 0) return VRC_ERR_INVALID;
    if (nq == 0) return VRC_OK;
    if (!d_q || !d_rgb || !d_status) return VRC_ERR_INVALID;
    vrc_grid* g = const_cast<vrc_grid*>(gc);   // query scratch lives in the grid object
    cudaStream_t st = (cudaStream_t)stream;
    if (g->q_cap < nq) {
        cudaFree(g->q_cell);
        cudaFree(g->q_rank);
        cudaFree(g->q_pts);
        g->q_cell = g->q_rank = nullptr;
        g->q_pts = nullptr;
        g->q_cap = 0;
        if (dev_alloc(&g->q_cell, nq) || dev_alloc(&g->q_rank, nq) || dev_alloc(&g->q_pts, nq)) return VRC_ERR_OOM;
        g->q_cap = nq;
    }
    int G = g->G, ncell = G * G * G;
    int tb = 256, nbk = (nq + tb - 1) / tb;
    VRC_CUDA_CHECK(cudaMemsetAsync(g->q_count, 0, sizeof(int) * (ncell + 1), st));
    k_bin_queries<<<nbk, tb, 0, st>>>(d_q, nq, G, g->q_cell, g->q_rank, g->q_count);
    // reuse cell_start-sized scratch: the query offsets go to q_count's scan in place
    int rc = exclusive_scan(g->q_count, ncell, g->q_count, g->scan_tmp, st);
    if (rc) return rc;
    k_scatter_queries<<<nbk, tb, 0, st>>>(d_q, g->q_cell, g->q_rank, g->q_count, nq, g->q_pts);
    auto kfn = g->order == 2 ? (g->aniso ? k_query<2, true> : k_query<2, false>)
                             : (g->aniso ? k_query<1, true> : k_query<1, false>);
    kfn<<<nbk, tb, 0, st>>>(g->rec, g->hess, g->ell, g->cell_start, g->cell_list, G, g->q_pts, nq, d_rgb,
                            d_status);
    return cudaGetLastError() == cudaSuccess ? VRC_OK : VRC_ERR_CUDA;
}
