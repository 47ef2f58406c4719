// noalloc.cu -- a query entry point that allocates nothing.
//
// vrc_query_inscatter needs a vrc_grid, which vrc_build_record_grid allocates with
// cudaMalloc (and which grows its query scratch on demand).  Some callers cannot do
// that: a host application or plugin framework that owns every byte of device memory
// and hands out fixed pools at start-up, a real-time renderer that forbids
// allocation after initialisation because cudaMalloc can synchronise the device and
// stall other streams, or a service that runs with a hard, pre-reserved memory
// budget.  vrc_query_inscatter_noalloc answers the same queries from the caller's
// record buffers with all of its working memory in one file-scope device array of
// fixed size, so it never calls cudaMalloc, cudaFree or an allocating library routine.
// It serves sphere records (the grids vrc_build_record_grid builds); the ellipsoid fields
// of the records (radii, axes) are not read.
//
// The working memory (VRC_NOALLOC_SCRATCH_INTS 32-bit words, 4 MiB) is a coarse
// 16 x 16 x 16 grid over the unit cube: per-cell counts, start offsets and the lists
// of records whose sphere of radius R_k overlaps each cell.  If the lists would not
// fit, the queries fall back to scanning every record (same results, slower).
// Every GPU that loads the library holds this array until the process exits.
#include <mutex>

#include "vrc_internal.cuh"

#define NA_G 16
#define NA_CELLS (NA_G * NA_G * NA_G)
#define NA_HEADER 16
// layout: header [16] | counts [NA_CELLS] | starts [NA_CELLS + 1] | lists [rest]
#define NA_LIST_OFFSET (NA_HEADER + NA_CELLS + NA_CELLS + 1 + 15)
#define NA_LIST_CAP (VRC_NOALLOC_SCRATCH_INTS - NA_LIST_OFFSET)

static __device__ __align__(256) int g_noalloc_scratch[VRC_NOALLOC_SCRATCH_INTS];

namespace {

std::mutex g_na_mutex;
int* g_na_ptr[64] = {nullptr};

// device address of g_noalloc_scratch on the current device (looked up once per device)
int na_scratch(int** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return VRC_ERR_CUDA;
    std::lock_guard<std::mutex> lock(g_na_mutex);
    if (!g_na_ptr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return VRC_ERR_CUDA;
        g_na_ptr[dev] = static_cast<int*>(p);
    }
    *out = g_na_ptr[dev];
    return VRC_OK;
}

__device__ __forceinline__ bool na_meets(float3 c, float R, int ix, int iy, int iz) {
    const float h = 1.0f / NA_G;
    float lx = ix * h, ly = iy * h, lz = iz * h;
    float dx = fmaxf(fmaxf(lx - c.x, c.x - (lx + h)), 0.f);
    float dy = fmaxf(fmaxf(ly - c.y, c.y - (ly + h)), 0.f);
    float dz = fmaxf(fmaxf(lz - c.z, c.z - (lz + h)), 0.f);
    return dx * dx + dy * dy + dz * dz < R * R;
}

__global__ void k_na_clear(int* s) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < NA_HEADER + NA_CELLS; i += gridDim.x * blockDim.x)
        s[i] = 0;
}

// FILL = false: count the cells each record's sphere overlaps; FILL = true: write the lists
template <bool FILL>
__global__ void k_na_insert(const float* pos, const float* radius, int n, int* s) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    int* counts = s + NA_HEADER;
    const int* starts = counts + NA_CELLS;
    int* list = s + NA_LIST_OFFSET;
    if (FILL && s[0]) return;                    // lists overflowed: queries scan all records
    float3 c = make_float3(pos[3 * k], pos[3 * k + 1], pos[3 * k + 2]);
    float R = radius[k];
    int x0 = max(0, (int)floorf((c.x - R) * NA_G)), x1 = min(NA_G - 1, (int)floorf((c.x + R) * NA_G));
    int y0 = max(0, (int)floorf((c.y - R) * NA_G)), y1 = min(NA_G - 1, (int)floorf((c.y + R) * NA_G));
    int z0 = max(0, (int)floorf((c.z - R) * NA_G)), z1 = min(NA_G - 1, (int)floorf((c.z + R) * NA_G));
    for (int ix = x0; ix <= x1; ++ix)
        for (int iy = y0; iy <= y1; ++iy)
            for (int iz = z0; iz <= z1; ++iz) {
                if (!na_meets(c, R, ix, iy, iz)) continue;
                int cell = (ix * NA_G + iy) * NA_G + iz;
                int slot = atomicAdd(&counts[cell], 1);
                if (FILL) list[starts[cell] + slot] = k;
            }
}

// one block: exclusive scan of the counts into starts, overflow flag, counts reset
__global__ void k_na_scan(int* s) {
    __shared__ int part[1024];
    int* counts = s + NA_HEADER;
    int* starts = counts + NA_CELLS;
    const int per = NA_CELLS / 1024;
    int t = threadIdx.x;
    int local = 0;
    for (int e = 0; e < per; ++e) local += counts[t * per + e];
    part[t] = local;
    __syncthreads();
    for (int off = 1; off < 1024; off <<= 1) {
        int v = t >= off ? part[t - off] : 0;
        __syncthreads();
        part[t] += v;
        __syncthreads();
    }
    int run = part[t] - local;
    for (int e = 0; e < per; ++e) {
        int i = t * per + e;
        starts[i] = run;
        run += counts[i];
        counts[i] = 0;                           // reused as fill cursors
    }
    if (t == 1023) {
        starts[NA_CELLS] = part[t];
        s[0] = part[t] > NA_LIST_CAP ? 1 : 0;
    }
}

// One block per cell puts the cell's list in ascending record order, so the queries sum
// their candidates in a fixed order.  The ids of a cell are distinct and below n <= 65,536:
// short lists are rank-sorted in shared memory; longer ones set one bit per id in a shared
// bitmap of n bits (8 KiB at most) and write the set bits back in order, O(len + n / 32).
#define NA_SORT_THREADS 256
#define NA_RANK_CAP 512
__global__ void __launch_bounds__(NA_SORT_THREADS) k_na_sort(int* s, int n) {
    __shared__ unsigned bits[VRC_NOALLOC_MAX_RECORDS / 32];
    __shared__ int part[NA_SORT_THREADS];
    const int cell = blockIdx.x, tid = threadIdx.x;
    if (s[0]) return;                            // overflowed: no lists
    const int* starts = s + NA_HEADER + NA_CELLS;
    int* list = s + NA_LIST_OFFSET;
    const int b = starts[cell], len = starts[cell + 1] - b;
    if (len <= 1) return;
    if (len <= NA_RANK_CAP) {
        int* buf = reinterpret_cast<int*>(bits);
        for (int i = tid; i < len; i += NA_SORT_THREADS) buf[i] = list[b + i];
        __syncthreads();
        for (int i = tid; i < len; i += NA_SORT_THREADS) {
            const int v = buf[i];
            int r = 0;
            for (int j = 0; j < len; ++j) r += buf[j] < v;
            list[b + r] = v;
        }
        return;
    }
    const int words = (n + 31) >> 5;
    for (int w = tid; w < words; w += NA_SORT_THREADS) bits[w] = 0u;
    __syncthreads();
    for (int i = tid; i < len; i += NA_SORT_THREADS) {
        const int id = list[b + i];
        atomicOr(&bits[id >> 5], 1u << (id & 31));
    }
    __syncthreads();
    // each thread owns a contiguous run of words; an exclusive scan of their bit counts
    // gives its first output slot
    const int per = (words + NA_SORT_THREADS - 1) / NA_SORT_THREADS;
    const int w0 = min(tid * per, words), w1 = min(w0 + per, words);
    int cnt = 0;
    for (int w = w0; w < w1; ++w) cnt += __popc(bits[w]);
    part[tid] = cnt;
    __syncthreads();
    for (int off = 1; off < NA_SORT_THREADS; off <<= 1) {
        const int t = tid >= off ? part[tid - off] : 0;
        __syncthreads();
        part[tid] += t;
        __syncthreads();
    }
    int o = b + part[tid] - cnt;
    for (int w = w0; w < w1; ++w) {
        unsigned m = bits[w];
        while (m) {
            list[o++] = (w << 5) + __ffs(m) - 1;
            m &= m - 1u;
        }
    }
}

// Eq. radianceTaylor for one query per thread, candidates in ascending record order
template <int ORDER>
__global__ void k_na_query(vrc_records_view v, int n, const int* s, const float* q, int nq, float* rgb,
                           int* status) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nq) return;
    float3 x = make_float3(q[3 * i], q[3 * i + 1], q[3 * i + 2]);
    bool all = s[0] != 0;
    int ix = min(NA_G - 1, max(0, (int)floorf(x.x * NA_G)));
    int iy = min(NA_G - 1, max(0, (int)floorf(x.y * NA_G)));
    int iz = min(NA_G - 1, max(0, (int)floorf(x.z * NA_G)));
    int cell = (ix * NA_G + iy) * NA_G + iz;
    const int* starts = s + NA_HEADER + NA_CELLS;
    const int* list = s + NA_LIST_OFFSET;
    int b = all ? 0 : starts[cell], e = all ? n : starts[cell + 1];
    float ar = 0.f, ag = 0.f, ab = 0.f, sw = 0.f;
    int cnt = 0;
    for (int p = b; p < e; ++p) {
        int k = all ? p : list[p];
        float px = v.pos[3 * k], py = v.pos[3 * k + 1], pz = v.pos[3 * k + 2], R = v.radius[k];
        float dx = x.x - px, dy = x.y - py, dz = x.z - pz;
        float d2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
        if (!(d2 < R * R)) continue;
        const float* L = v.L + 3 * k;
        const float* g = v.grad + 9 * k;
        float dd = 1.0f - sqrtf(d2) / R;
        float w = dd * dd * fmaf(-2.0f, dd, 3.0f);
        float vr = L[0] + fmaf(g[0], dx, fmaf(g[1], dy, g[2] * dz));
        float vg = L[1] + fmaf(g[3], dx, fmaf(g[4], dy, g[5] * dz));
        float vb = L[2] + fmaf(g[6], dx, fmaf(g[7], dy, g[8] * dz));
        if (ORDER == 2) {
            const float* hh = v.hess + 18 * k;
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
    }
    float inv = cnt ? 1.0f / sw : 0.0f;
    rgb[3 * i] = ar * inv;
    rgb[3 * i + 1] = ag * inv;
    rgb[3 * i + 2] = ab * inv;
    status[i] = cnt;
}

}  // namespace

extern "C" int vrc_query_inscatter_noalloc(const vrc_records_view* recs, int32_t n, int32_t extrap_order,
                                           const float* d_q, int32_t nq, float* d_rgb, int32_t* d_status,
                                           void* stream) {
    if (!recs || n < 0 || nq < 0 || (extrap_order != 1 && extrap_order != 2)) return VRC_ERR_INVALID;
    if (n > VRC_NOALLOC_MAX_RECORDS) return VRC_ERR_UNSUPPORTED;
    if (nq == 0) return VRC_OK;
    if (!d_q || !d_rgb || !d_status) return VRC_ERR_INVALID;
    if (n > 0 && (!recs->pos || !recs->radius || !recs->L || !recs->grad || (extrap_order == 2 && !recs->hess)))
        return VRC_ERR_INVALID;
    int* s = nullptr;
    int rc = na_scratch(&s);
    if (rc != VRC_OK) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    k_na_clear<<<16, 256, 0, st>>>(s);
    if (n > 0) {
        int nb = (n + 255) / 256;
        k_na_insert<false><<<nb, 256, 0, st>>>(recs->pos, recs->radius, n, s);
        k_na_scan<<<1, 1024, 0, st>>>(s);
        k_na_insert<true><<<nb, 256, 0, st>>>(recs->pos, recs->radius, n, s);
        k_na_sort<<<NA_CELLS, NA_SORT_THREADS, 0, st>>>(s, n);
    } else {
        k_na_scan<<<1, 1024, 0, st>>>(s);
    }
    int qb = (nq + 255) / 256;
    if (extrap_order == 2)
        k_na_query<2><<<qb, 256, 0, st>>>(*recs, n, s, d_q, nq, d_rgb, d_status);
    else
        k_na_query<1><<<qb, 256, 0, st>>>(*recs, n, s, d_q, nq, d_rgb, d_status);
    return cudaGetLastError() == cudaSuccess ? VRC_OK : VRC_ERR_CUDA;
}
