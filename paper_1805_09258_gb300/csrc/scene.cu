// scene.cu -- scene upload and bounding volume hierarchy (host build, device layout).
//
// The paper traces its ray sets with Embree on a CPU (Sec. 6); here the scene lives
// in HBM as a two-wide BVH built on the host with binned surface-area heuristic
// splits, traversed by the library's own kernels (vrc_internal.cuh).
#include <algorithm>
#include <array>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <limits>
#include <vector>

#include "vrc_internal.cuh"

namespace {

struct BTri {
    float lo[3], hi[3], c[3];
    int id;
};

struct HNode {
    float lo[2][3], hi[2][3];
    int child[2];
};

struct Builder {
    std::vector<BTri> tris;
    std::vector<HNode> nodes;
    std::vector<int> order;   // leaf order of original triangle ids
    int max_depth = 0;

    static void bound(const BTri* t, int n, float lo[3], float hi[3]) {
        for (int k = 0; k < 3; ++k) { lo[k] = 1e30f; hi[k] = -1e30f; }
        for (int i = 0; i < n; ++i)
            for (int k = 0; k < 3; ++k) {
                lo[k] = std::min(lo[k], t[i].lo[k]);
                hi[k] = std::max(hi[k], t[i].hi[k]);
            }
    }
    static float area(const float lo[3], const float hi[3]) {
        float dx = std::max(0.f, hi[0] - lo[0]), dy = std::max(0.f, hi[1] - lo[1]), dz = std::max(0.f, hi[2] - lo[2]);
        return 2.f * (dx * dy + dy * dz + dz * dx);
    }

    int make_leaf(int begin, int count) {
        int first = (int)order.size();
        for (int i = begin; i < begin + count; ++i) order.push_back(tris[i].id);
        return -(1 + ((first << 3) | (count - 1)));
    }

    // returns a child code for tris[begin, begin + count)
    int build(int begin, int count, int depth) {
        max_depth = std::max(max_depth, depth);
        if (count <= 2) return make_leaf(begin, count);
        float clo[3] = {1e30f, 1e30f, 1e30f}, chi[3] = {-1e30f, -1e30f, -1e30f};
        for (int i = begin; i < begin + count; ++i)
            for (int k = 0; k < 3; ++k) {
                clo[k] = std::min(clo[k], tris[i].c[k]);
                chi[k] = std::max(chi[k], tris[i].c[k]);
            }
        const int NB = 16;
        float best_cost = 1e30f;
        int best_axis = -1, best_bin = -1;
        float plo[3], phi[3];
        bound(&tris[begin], count, plo, phi);
        float parea = std::max(area(plo, phi), 1e-30f);
        for (int ax = 0; ax < 3; ++ax) {
            float ext = chi[ax] - clo[ax];
            if (!(ext > 0.f)) continue;
            int cnt[NB] = {0};
            float blo[NB][3], bhi[NB][3];
            for (int b = 0; b < NB; ++b)
                for (int k = 0; k < 3; ++k) { blo[b][k] = 1e30f; bhi[b][k] = -1e30f; }
            for (int i = begin; i < begin + count; ++i) {
                int b = std::min(NB - 1, (int)((tris[i].c[ax] - clo[ax]) / ext * NB));
                cnt[b]++;
                for (int k = 0; k < 3; ++k) {
                    blo[b][k] = std::min(blo[b][k], tris[i].lo[k]);
                    bhi[b][k] = std::max(bhi[b][k], tris[i].hi[k]);
                }
            }
            float rlo[NB][3], rhi[NB][3];
            int rcnt[NB];
            float alo[3] = {1e30f, 1e30f, 1e30f}, ahi[3] = {-1e30f, -1e30f, -1e30f};
            int acc = 0;
            for (int b = NB - 1; b >= 0; --b) {
                for (int k = 0; k < 3; ++k) { alo[k] = std::min(alo[k], blo[b][k]); ahi[k] = std::max(ahi[k], bhi[b][k]); }
                acc += cnt[b];
                std::memcpy(rlo[b], alo, sizeof(alo));
                std::memcpy(rhi[b], ahi, sizeof(ahi));
                rcnt[b] = acc;
            }
            for (int k = 0; k < 3; ++k) { alo[k] = 1e30f; ahi[k] = -1e30f; }
            acc = 0;
            for (int b = 0; b < NB - 1; ++b) {
                for (int k = 0; k < 3; ++k) { alo[k] = std::min(alo[k], blo[b][k]); ahi[k] = std::max(ahi[k], bhi[b][k]); }
                acc += cnt[b];
                if (acc == 0 || rcnt[b + 1] == 0) continue;
                float cost = 0.125f + (area(alo, ahi) * acc + area(rlo[b + 1], rhi[b + 1]) * rcnt[b + 1]) / parea;
                if (cost < best_cost) { best_cost = cost; best_axis = ax; best_bin = b; }
            }
        }
        int mid;
        if (best_axis < 0) {
            if (count <= 8) return make_leaf(begin, count);
            mid = begin + count / 2;    // all centroids coincide: split by index
        } else {
            if (count <= 4 && best_cost >= (float)count) return make_leaf(begin, count);
            float ext = chi[best_axis] - clo[best_axis];
            auto it = std::partition(tris.begin() + begin, tris.begin() + begin + count, [&](const BTri& t) {
                int b = std::min(NB - 1, (int)((t.c[best_axis] - clo[best_axis]) / ext * NB));
                return b <= best_bin;
            });
            mid = (int)(it - tris.begin());
            if (mid == begin || mid == begin + count) mid = begin + count / 2;
        }
        int me = (int)nodes.size();
        nodes.push_back(HNode());
        int c0 = build(begin, mid - begin, depth + 1);
        int c1 = build(mid, begin + count - mid, depth + 1);
        HNode& nd = nodes[me];
        bound(&tris[begin], mid - begin, nd.lo[0], nd.hi[0]);
        bound(&tris[mid], begin + count - mid, nd.lo[1], nd.hi[1]);
        nd.child[0] = c0;
        nd.child[1] = c1;
        return me;
    }
};

float bits_as_float(int v) {
    float f;
    std::memcpy(&f, &v, sizeof(f));
    return f;
}

// ---------------------------------------------------------------- light buffer
// For each cube face around the light (face = 2 axis + (negative ? 1 : 0); coordinates
// m along the axis, a and b the next two axes cyclically) the triangle is clipped to the
// face's frustum m >= |a|, m >= |b| (Sutherland-Hodgman), projected to (a/m, b/m), and its
// padded bounding rectangle of cells receives the triangle.  The gnomonic projection maps
// the clipped polygon onto a convex polygon inside that rectangle, so every direction the
// triangle covers (and a margin for rounding and for the widened triangle test) lands in
// a cell that lists it.  Entries of a cell are sorted by a lower bound of the triangle's
// distance to the light: the larger of the distance to its bounding box and its distance
// inside the cell's padded frustum (a triangle with no part there is left out).  Each cell
// also records the bound of its first entry, and the covered distance: the smallest, over the
// cell's triangles that every direction of the cell crosses (the four corner rays hit it with
// barycentrics at least 1e-3 inside its edges, at least 0.06 degrees off its plane), of the
// largest corner hit distance, padded for the float ray test.
struct LightBufHost {
    std::vector<int4> cell;
    std::vector<int2> ent;
};

// Whether the four corner rays from the light (directions dir, not normalised) all cross
// triangle T (vertices relative to the light) well inside it; hmax gets the largest hit
// distance.  Double precision.
static bool covers_cell(const double q[3][3], const double dir[4][3], double& hmax) {
    const double mb = 1e-3;
    double e1[3], e2[3], nrm[3];
    for (int k = 0; k < 3; ++k) {
        e1[k] = q[1][k] - q[0][k];
        e2[k] = q[2][k] - q[0][k];
    }
    nrm[0] = e1[1] * e2[2] - e1[2] * e2[1];
    nrm[1] = e1[2] * e2[0] - e1[0] * e2[2];
    nrm[2] = e1[0] * e2[1] - e1[1] * e2[0];
    const double nn = std::sqrt(nrm[0] * nrm[0] + nrm[1] * nrm[1] + nrm[2] * nrm[2]);
    if (!(nn > 0.0)) return false;
    hmax = 0.0;
    for (int c = 0; c < 4; ++c) {
        const double* d = dir[c];
        const double dn = std::sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
        if (std::fabs(d[0] * nrm[0] + d[1] * nrm[1] + d[2] * nrm[2]) < 1e-3 * dn * nn) return false;
        double p[3] = {d[1] * e2[2] - d[2] * e2[1], d[2] * e2[0] - d[0] * e2[2], d[0] * e2[1] - d[1] * e2[0]};
        const double det = e1[0] * p[0] + e1[1] * p[1] + e1[2] * p[2];
        const double s[3] = {-q[0][0], -q[0][1], -q[0][2]};       // the light relative to vertex 0
        const double u = (s[0] * p[0] + s[1] * p[1] + s[2] * p[2]) / det;
        const double qv[3] = {s[1] * e1[2] - s[2] * e1[1], s[2] * e1[0] - s[0] * e1[2], s[0] * e1[1] - s[1] * e1[0]};
        const double v = (d[0] * qv[0] + d[1] * qv[1] + d[2] * qv[2]) / det;
        const double t = (e2[0] * qv[0] + e2[1] * qv[1] + e2[2] * qv[2]) / det;
        if (!(u >= mb && v >= mb && u + v <= 1.0 - mb && t > 0.0)) return false;
        hmax = std::max(hmax, t * dn);
    }
    return true;
}

// The part of triangle T (vertices as (m, a, b) relative to the light) inside the frustum
// u0 <= a/m <= u1, v0 <= b/m <= v1: false if none, else md gets its distance to the light.
// Double precision.
static bool cell_distance(const double T[3][3], double u0, double u1, double v0, double v1, double& md) {
    double P[12][3], Q[12][3];
    int n = 3;
    for (int v = 0; v < 3; ++v)
        for (int k = 0; k < 3; ++k) P[v][k] = T[v][k];
    // half-spaces a - u0 m >= 0, u1 m - a >= 0, b - v0 m >= 0, v1 m - b >= 0
    const double pl[4][3] = {{-u0, 1, 0}, {u1, -1, 0}, {-v0, 0, 1}, {v1, 0, -1}};
    for (int p = 0; p < 4 && n > 0; ++p) {
        int o = 0;
        for (int i = 0; i < n; ++i) {
            const double* A = P[i];
            const double* B = P[(i + 1) % n];
            double da = pl[p][0] * A[0] + pl[p][1] * A[1] + pl[p][2] * A[2];
            double db = pl[p][0] * B[0] + pl[p][1] * B[1] + pl[p][2] * B[2];
            if (da >= 0) {
                for (int k = 0; k < 3; ++k) Q[o][k] = A[k];
                ++o;
            }
            if ((da >= 0) != (db >= 0)) {
                double s2 = da / (da - db);
                for (int k = 0; k < 3; ++k) Q[o][k] = A[k] + s2 * (B[k] - A[k]);
                ++o;
            }
        }
        n = o;
        for (int i = 0; i < n; ++i)
            for (int k = 0; k < 3; ++k) P[i][k] = Q[i][k];
    }
    if (n == 0) return false;
    // nearest point of the convex polygon to the light: the foot of the perpendicular when it
    // falls inside, else the nearest point of an edge
    double e1[3], e2[3], nr[3];
    for (int k = 0; k < 3; ++k) {
        e1[k] = T[1][k] - T[0][k];
        e2[k] = T[2][k] - T[0][k];
    }
    nr[0] = e1[1] * e2[2] - e1[2] * e2[1];
    nr[1] = e1[2] * e2[0] - e1[0] * e2[2];
    nr[2] = e1[0] * e2[1] - e1[1] * e2[0];
    const double nn = nr[0] * nr[0] + nr[1] * nr[1] + nr[2] * nr[2];
    double best = 1e300;
    if (nn > 0.0 && n >= 3) {
        const double h = (nr[0] * T[0][0] + nr[1] * T[0][1] + nr[2] * T[0][2]) / nn;
        const double f[3] = {h * nr[0], h * nr[1], h * nr[2]};
        bool pos = true, neg = true;
        for (int i = 0; i < n; ++i) {
            const double* A = P[i];
            const double* B = P[(i + 1) % n];
            double ex[3] = {B[0] - A[0], B[1] - A[1], B[2] - A[2]};
            double fx[3] = {f[0] - A[0], f[1] - A[1], f[2] - A[2]};
            double c = nr[0] * (ex[1] * fx[2] - ex[2] * fx[1]) + nr[1] * (ex[2] * fx[0] - ex[0] * fx[2]) +
                       nr[2] * (ex[0] * fx[1] - ex[1] * fx[0]);
            if (c < 0) pos = false;
            if (c > 0) neg = false;
        }
        if (pos || neg) best = std::sqrt(f[0] * f[0] + f[1] * f[1] + f[2] * f[2]);
    }
    for (int i = 0; i < n; ++i) {
        const double* A = P[i];
        const double* B = P[(i + 1) % n];
        double ex[3] = {B[0] - A[0], B[1] - A[1], B[2] - A[2]};
        double ee = ex[0] * ex[0] + ex[1] * ex[1] + ex[2] * ex[2];
        double s2 = ee > 0.0 ? -(A[0] * ex[0] + A[1] * ex[1] + A[2] * ex[2]) / ee : 0.0;
        s2 = std::min(1.0, std::max(0.0, s2));
        double x[3] = {A[0] + s2 * ex[0], A[1] + s2 * ex[1], A[2] + s2 * ex[2]};
        best = std::min(best, std::sqrt(x[0] * x[0] + x[1] * x[1] + x[2] * x[2]));
    }
    md = best;
    return true;
}

void build_light_buffer(const std::vector<std::array<double, 9>>& tv, const std::vector<int>& bvh_index,
                        const double L[3], int R, LightBufHost& out) {
    const int ncell = 6 * R * R;
    std::vector<std::vector<std::pair<float, int>>> cells(ncell);
    std::vector<int> orig(tv.size());                 // BVH leaf order -> triangle
    const double pad = 1e-4;
    for (size_t t = 0; t < tv.size(); ++t) {
        double q[3][3];
        double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
        for (int v = 0; v < 3; ++v)
            for (int k = 0; k < 3; ++k) {
                q[v][k] = tv[t][3 * v + k] - L[k];
                lo[k] = std::min(lo[k], tv[t][3 * v + k]);
                hi[k] = std::max(hi[k], tv[t][3 * v + k]);
            }
        orig[bvh_index[t]] = (int)t;
        double dd = 0.0;
        for (int k = 0; k < 3; ++k) {
            double e = std::max(std::max(lo[k] - L[k], L[k] - hi[k]), 0.0);
            dd += e * e;
        }
        float dmin = (float)(std::sqrt(dd) * (1.0 - 1e-6));
        dmin = std::nextafter(dmin, 0.0f);
        for (int face = 0; face < 6; ++face) {
            int axis = face / 2;
            double sg = (face & 1) ? -1.0 : 1.0;
            int ia = (axis + 1) % 3, ib = (axis + 2) % 3;
            std::vector<std::array<double, 3>> poly;   // (m, a, b)
            for (int v = 0; v < 3; ++v) poly.push_back({sg * q[v][axis], q[v][ia], q[v][ib]});
            // clip against m - a >= 0, m + a >= 0, m - b >= 0, m + b >= 0
            const double pl[4][3] = {{1, -1, 0}, {1, 1, 0}, {1, 0, -1}, {1, 0, 1}};
            for (int p = 0; p < 4 && !poly.empty(); ++p) {
                std::vector<std::array<double, 3>> o;
                size_t n = poly.size();
                for (size_t i = 0; i < n; ++i) {
                    const auto& A = poly[i];
                    const auto& B = poly[(i + 1) % n];
                    double da = pl[p][0] * A[0] + pl[p][1] * A[1] + pl[p][2] * A[2];
                    double db = pl[p][0] * B[0] + pl[p][1] * B[1] + pl[p][2] * B[2];
                    if (da >= 0) o.push_back(A);
                    if ((da >= 0) != (db >= 0)) {
                        double s2 = da / (da - db);
                        o.push_back({A[0] + s2 * (B[0] - A[0]), A[1] + s2 * (B[1] - A[1]), A[2] + s2 * (B[2] - A[2])});
                    }
                }
                poly.swap(o);
            }
            if (poly.empty()) continue;
            double umin = 1e300, umax = -1e300, vmin = 1e300, vmax = -1e300;
            bool apex = false;
            for (const auto& P : poly) {
                if (P[0] <= 1e-12) { apex = true; break; }
                double u = P[1] / P[0], v = P[2] / P[0];
                umin = std::min(umin, u); umax = std::max(umax, u);
                vmin = std::min(vmin, v); vmax = std::max(vmax, v);
            }
            if (apex) { umin = vmin = -1.0; umax = vmax = 1.0; }
            auto cidx = [&](double u) { return std::min(R - 1, std::max(0, (int)std::floor((u + 1.0) * 0.5 * R))); };
            int i0 = cidx(umin - pad), i1 = cidx(umax + pad), j0 = cidx(vmin - pad), j1 = cidx(vmax + pad);
            double tri[3][3];
            for (int v = 0; v < 3; ++v) {
                tri[v][0] = sg * q[v][axis];
                tri[v][1] = q[v][ia];
                tri[v][2] = q[v][ib];
            }
            for (int i = i0; i <= i1; ++i)
                for (int j = j0; j <= j1; ++j) {
                    // the triangle within the cell's padded frustum: no part, no entry; else
                    // its distance there, less a margin for the widened float ray test, is
                    // the entry's bound when it beats the bounding-box one
                    double md;
                    if (!cell_distance(tri, 2.0 * i / R - 1.0 - pad, 2.0 * (i + 1) / R - 1.0 + pad,
                                       2.0 * j / R - 1.0 - pad, 2.0 * (j + 1) / R - 1.0 + pad, md))
                        continue;
                    float bd = (float)(md * (1.0 - 1e-5) - 1e-6);
                    bd = std::nextafter(bd, 0.0f);
                    cells[(face * R + i) * R + j].push_back({std::max(dmin, bd), bvh_index[t]});
                }
        }
    }
    out.cell.assign(ncell, make_int4(0, 0, 0, 0));
    size_t total = 0;
    for (int c = 0; c < ncell; ++c) total += cells[c].size();
    out.ent.resize(total);
    const float inf = std::numeric_limits<float>::infinity();
    size_t at = 0;
    for (int c = 0; c < ncell; ++c) {
        auto& v = cells[c];
        std::sort(v.begin(), v.end());
        for (size_t k = 0; k < v.size(); ++k) {
            int bits;
            std::memcpy(&bits, &v[k].first, sizeof(bits));
            out.ent[at + k] = make_int2(v[k].second, bits);
        }
        // corner directions of the cell: major axis +-1, the next two axes at the cell's edges
        const int face = c / (R * R), i = (c / R) % R, j = c % R;
        const int axis = face / 2, ia = (axis + 1) % 3, ib = (axis + 2) % 3;
        const double sg = (face & 1) ? -1.0 : 1.0;
        double dir[4][3];
        for (int k = 0; k < 4; ++k) {
            dir[k][axis] = sg;
            dir[k][ia] = 2.0 * (i + (k & 1)) / R - 1.0;
            dir[k][ib] = 2.0 * (j + (k >> 1)) / R - 1.0;
        }
        double dsh = std::numeric_limits<double>::infinity();
        for (size_t k = 0; k < v.size() && (double)v[k].first < dsh; ++k) {
            const auto& T = tv[orig[v[k].second]];
            double q[3][3];
            for (int a = 0; a < 3; ++a)
                for (int b = 0; b < 3; ++b) q[a][b] = T[3 * a + b] - L[b];
            double hmax;
            if (covers_cell(q, dir, hmax)) dsh = std::min(dsh, hmax * (1.0 + 1e-4) + 1e-5);
        }
        float dfirst = v.empty() ? inf : v[0].first;
        float fsh = std::isinf(dsh) ? inf : std::nextafter((float)dsh, inf);
        int bf, bs;
        std::memcpy(&bf, &dfirst, sizeof(bf));
        std::memcpy(&bs, &fsh, sizeof(bs));
        out.cell[c] = make_int4((int)at, (int)(at + v.size()), bf, bs);
        at += v.size();
    }
}

int upload(void** dst, const void* src, size_t bytes) {
    if (cudaMalloc(dst, bytes == 0 ? 16 : bytes) != cudaSuccess) return VRC_ERR_OOM;
    if (bytes && cudaMemcpy(*dst, src, bytes, cudaMemcpyHostToDevice) != cudaSuccess) return VRC_ERR_CUDA;
    return VRC_OK;
}

}  // namespace

extern "C" int vrc_build_scene(const float* verts, int32_t n_verts, const int32_t* idx, int32_t n_tris,
                               const float* albedo, const float* emission, const vrc_medium* medium,
                               const vrc_point_light* lights, int32_t n_lights, vrc_scene** out) {
    if (!out || !medium || n_tris < 0 || n_verts < 0 || n_lights < 0 || n_lights > VRC_MAX_LIGHTS)
        return VRC_ERR_INVALID;
    if (n_tris > 0 && (!verts || !idx || !albedo)) return VRC_ERR_INVALID;
    if (n_lights > 0 && !lights) return VRC_ERR_INVALID;
    if (n_tris >= (1 << 27)) return VRC_ERR_UNSUPPORTED;
    *out = nullptr;
    Builder B;
    B.tris.resize(n_tris);
    std::vector<float4> prim(3 * (size_t)std::max(n_tris, 1));
    for (int t = 0; t < n_tris; ++t) {
        double p[3][3];
        for (int q = 0; q < 3; ++q) {
            int vi = idx[3 * t + q];
            if (vi < 0 || vi >= n_verts) return VRC_ERR_INVALID;
            for (int k = 0; k < 3; ++k) p[q][k] = (double)verts[3 * vi + k];
        }
        BTri& bt = B.tris[t];
        for (int k = 0; k < 3; ++k) {
            bt.lo[k] = (float)std::min(p[0][k], std::min(p[1][k], p[2][k]));
            bt.hi[k] = (float)std::max(p[0][k], std::max(p[1][k], p[2][k]));
            bt.c[k] = (float)((p[0][k] + p[1][k] + p[2][k]) / 3.0);
        }
        bt.id = t;
        double e1[3], e2[3], n[3];
        for (int k = 0; k < 3; ++k) { e1[k] = p[1][k] - p[0][k]; e2[k] = p[2][k] - p[0][k]; }
        n[0] = e1[1] * e2[2] - e1[2] * e2[1];
        n[1] = e1[2] * e2[0] - e1[0] * e2[2];
        n[2] = e1[0] * e2[1] - e1[1] * e2[0];
        double nl = std::sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
        if (!(nl > 0.0)) nl = 1.0;   // zero-area triangle: never hit, normal unused
        prim[3 * t] = make_float4((float)(n[0] / nl), (float)(n[1] / nl), (float)(n[2] / nl), 0.f);
        prim[3 * t + 1] = make_float4(albedo[3 * t], albedo[3 * t + 1], albedo[3 * t + 2], 0.f);
        prim[3 * t + 2] = emission ? make_float4(emission[3 * t], emission[3 * t + 1], emission[3 * t + 2], 0.f)
                                   : make_float4(0.f, 0.f, 0.f, 0.f);
    }
    // root is always an inner node; a scene of <= 2 triangles gets an unreachable
    // second child (a point box far outside the unit cube)
    std::vector<float4> nodes;
    std::vector<float4> tris;
    if (n_tris > 0) {
        B.nodes.reserve(2 * (size_t)n_tris);
        int root = B.build(0, n_tris, 0);
        if (B.max_depth >= VRC_STACK - 2) return VRC_ERR_UNSUPPORTED;
        if (root < 0) {
            HNode r;
            Builder::bound(B.tris.data(), n_tris, r.lo[0], r.hi[0]);
            for (int k = 0; k < 3; ++k) { r.lo[1][k] = 1e30f; r.hi[1][k] = 1e30f; }
            r.child[0] = root;
            r.child[1] = root;
            B.nodes.insert(B.nodes.begin(), r);   // no inner indices to fix: the only child is a leaf
        }
        nodes.resize(4 * B.nodes.size());
        for (size_t i = 0; i < B.nodes.size(); ++i) {
            const HNode& h = B.nodes[i];
            nodes[4 * i] = make_float4(h.lo[0][0], h.hi[0][0], h.lo[0][1], h.hi[0][1]);
            nodes[4 * i + 1] = make_float4(h.lo[1][0], h.hi[1][0], h.lo[1][1], h.hi[1][1]);
            nodes[4 * i + 2] = make_float4(h.lo[0][2], h.hi[0][2], h.lo[1][2], h.hi[1][2]);
            nodes[4 * i + 3] = make_float4(bits_as_float(h.child[0]), bits_as_float(h.child[1]), 0.f, 0.f);
        }
        tris.resize(3 * (size_t)n_tris);
        for (int k = 0; k < n_tris; ++k) {
            int t = B.order[k];
            double p[3][3];
            for (int q = 0; q < 3; ++q)
                for (int c = 0; c < 3; ++c) p[q][c] = (double)verts[3 * idx[3 * t + q] + c];
            tris[3 * k] = make_float4((float)p[0][0], (float)p[0][1], (float)p[0][2], bits_as_float(t));
            tris[3 * k + 1] = make_float4((float)(p[1][0] - p[0][0]), (float)(p[1][1] - p[0][1]),
                                          (float)(p[1][2] - p[0][2]), 0.f);
            tris[3 * k + 2] = make_float4((float)(p[2][0] - p[0][0]), (float)(p[2][1] - p[0][1]),
                                          (float)(p[2][2] - p[0][2]), 0.f);
        }
    }
    // light buffers: triangle vertices in original order, mapped to BVH leaf order
    std::vector<LightBufHost> lbs(n_lights);
    // cube-map resolution: 256 x 256 cells per face (a 0.35 degree cell).  Measured against 64 /
    // 128: 2 % faster records on a 2,048-triangle scene, 10 % on a 250,000-triangle one, for a
    // few MB more per light and no slower build
    const int lbR = 256;
    if (n_tris > 0 && n_lights > 0) {
        std::vector<std::array<double, 9>> tv(n_tris);
        std::vector<int> bvh_index(n_tris);
        for (int k = 0; k < n_tris; ++k) bvh_index[B.order[k]] = k;
        for (int t = 0; t < n_tris; ++t)
            for (int q = 0; q < 3; ++q)
                for (int c = 0; c < 3; ++c) tv[t][3 * q + c] = (double)verts[3 * idx[3 * t + q] + c];
        for (int l = 0; l < n_lights; ++l) {
            double L[3] = {lights[l].pos[0], lights[l].pos[1], lights[l].pos[2]};
            build_light_buffer(tv, bvh_index, L, lbR, lbs[l]);
        }
    }
    vrc_scene* s = (vrc_scene*)std::calloc(1, sizeof(vrc_scene));
    if (!s) return VRC_ERR_OOM;
    int rc = VRC_OK;
    for (int l = 0; l < n_lights; ++l) {
        if (lbs[l].cell.empty()) {
            const float inf = std::numeric_limits<float>::infinity();
            int bi;
            std::memcpy(&bi, &inf, sizeof(bi));
            lbs[l].cell.assign(6 * lbR * lbR, make_int4(0, 0, bi, bi));
        }
        if ((rc = upload((void**)&s->d_lb_cell[l], lbs[l].cell.data(), lbs[l].cell.size() * sizeof(int4))) ||
            (rc = upload((void**)&s->d_lb_ent[l], lbs[l].ent.data(), lbs[l].ent.size() * sizeof(int2)))) {
            vrc_destroy_scene(s);
            return rc;
        }
        s->lb_entries += (long long)lbs[l].ent.size();
    }
    if ((rc = upload((void**)&s->d_nodes, nodes.data(), nodes.size() * sizeof(float4))) ||
        (rc = upload((void**)&s->d_tris, tris.data(), tris.size() * sizeof(float4))) ||
        (rc = upload((void**)&s->d_prim, prim.data(), prim.size() * sizeof(float4)))) {
        vrc_destroy_scene(s);
        return rc;
    }
    if (cudaMalloc((void**)&s->d_counter, 64) != cudaSuccess) {
        vrc_destroy_scene(s);
        return VRC_ERR_OOM;
    }
    s->n_prims = n_tris;
    DevScene& d = s->dev;
    d.nodes = s->d_nodes;
    d.tris = s->d_tris;
    d.prim = s->d_prim;
    d.n_nodes = (int)(nodes.size() / 4);
    d.n_tris = n_tris;
    d.n_lights = n_lights;
    for (int l = 0; l < n_lights; ++l) {
        d.lpos[l] = make_float3(lights[l].pos[0], lights[l].pos[1], lights[l].pos[2]);
        d.lI[l] = make_float3(lights[l].intensity[0], lights[l].intensity[1], lights[l].intensity[2]);
        d.lb[l].cell = s->d_lb_cell[l];
        d.lb[l].ent = s->d_lb_ent[l];
        d.lb[l].R = lbR;
    }
    d.use_lb = 1;
    d.sigma_s = medium->sigma_s;
    d.sigma_t = medium->sigma_s + medium->sigma_a;
    d.g = medium->g;
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&s->sm_count, cudaDevAttrMultiProcessorCount, dev);
    *out = s;
    return VRC_OK;
}

extern "C" void vrc_destroy_scene(vrc_scene* s) {
    if (!s) return;
    cudaFree(s->d_nodes);
    cudaFree(s->d_tris);
    cudaFree(s->d_prim);
    cudaFree(s->d_counter);
    cudaFree(s->d_order);
    for (int i = 0; i < s->t_ev_made; ++i)
        for (int e = 0; e < 4; ++e) cudaEventDestroy(s->t_ev[i][e]);
    cudaFree(s->d_pre_ray);
    cudaFree(s->d_pre_Lo);
    cudaFree(s->h_stage_dev);
    cudaFree(s->q_stage_dev);
    if (s->step_made) {
        for (int i = 0; i < 2; ++i) {
            cudaStreamDestroy(s->step_st[i]);
            cudaEventDestroy(s->step_ev[i]);
        }
    }
    for (int l = 0; l < VRC_MAX_LIGHTS; ++l) {
        cudaFree(s->d_lb_cell[l]);
        cudaFree(s->d_lb_ent[l]);
    }
    std::free(s);
}

extern "C" const char* vrc_status_string(int st) {
    switch (st) {
        case VRC_OK: return "ok";
        case VRC_ERR_INVALID: return "invalid argument";
        case VRC_ERR_OOM: return "out of memory";
        case VRC_ERR_CUDA: return "CUDA error";
        case VRC_ERR_TIMEOUT: return "device wait timed out";
        case VRC_ERR_UNSUPPORTED: return "unsupported size";
        default: return "unknown status";
    }
}

extern "C" int vrc_version(void) { return 100; }
