/*
 * vrc.h -- C ABI of the GB300 (sm_103a) library for second-order occlusion-aware
 * volumetric radiance caching (Marco, Jarabo, Jarosz, Gutierrez, "Second-Order
 * Occlusion-Aware Volumetric Radiance Caching", ACM TOG 37(2), 2018).
 *
 * The library computes cache records -- in-scattered radiance L together with its
 * occlusion-aware translational gradient and Hessian at a point x of a homogeneous
 * medium -- and answers interpolation queries from them.  Every step runs in the
 * library's own CUDA kernels; there is no CPU fallback.
 *
 * Conventions shared by all calls
 *   - The participating medium fills the unit cube [0,1]^3; all geometry lies in it.
 *   - Pointers named d_* are DEVICE pointers owned by the caller; other pointers
 *     are host pointers, read during the call only.  Opaque objects (vrc_scene,
 *     vrc_grid, vrc_mlp) are owned by the library and freed by their destroy call.
 *   - `stream` is a cudaStream_t passed as void* (0 = the legacy default stream).
 *     Calls that take a stream are asynchronous on it unless documented otherwise.
 *   - Every call returns an int status: VRC_OK (0) or a negative VRC_ERR_* code;
 *     vrc_status_string() names it.  No C++ exception crosses the ABI.  Per-item
 *     outcomes (a record whose radius was clamped, a query that found no record)
 *     go to caller-provided status arrays.
 *   - Vectors are float32 xyz; RGB triples are float32 r,g,b.  A gradient of an
 *     RGB quantity is stored [channel][axis] (9 floats), a Hessian [channel][6]
 *     with the 6 unique entries in the order xx, xy, xz, yy, yz, zz (18 floats).
 */
#ifndef VRC_H
#define VRC_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------ status codes */
#define VRC_OK 0
#define VRC_ERR_INVALID -1      /* a null pointer, size or parameter out of range */
#define VRC_ERR_OOM -2          /* a device or host allocation failed */
#define VRC_ERR_CUDA -3         /* a CUDA runtime call failed (launch, copy) */
#define VRC_ERR_TIMEOUT -4      /* a bounded device-side wait gave up */
#define VRC_ERR_UNSUPPORTED -5  /* a size beyond what the kernels handle */

/* per-record status bits (vrc_records_view.status) */
#define VRC_REC_NONFINITE 1     /* a non-finite value was produced */
#define VRC_REC_CLAMP_LO 2      /* radius clamped to r_min (or L <= 0) */
#define VRC_REC_CLAMP_HI 4      /* radius clamped to r_max (or a zero Hessian) */
#define VRC_REC_DEGENERATE 8    /* at least one cell had A = B = 0 and was skipped */
#define VRC_REC_BAD_COUNT 16    /* per-record band count outside [2, params n_bands]: not computed */

/* --------------------------------------------------------------- scene */
/* Homogeneous medium (Sec. 3, Table 1): scattering and absorption coefficients and
 * the Henyey-Greenstein asymmetry g of the phase function. */
typedef struct { float sigma_s, sigma_a, g; } vrc_medium;

/* Point light (handled by shadow rays, Sec. 6 "Implementation"). */
typedef struct { float pos[3]; float intensity[3]; } vrc_point_light;

#define VRC_MAX_LIGHTS 4

typedef struct vrc_scene vrc_scene;
typedef struct vrc_grid vrc_grid;   /* record lookup structure (vrc_build_record_grid) */

/* Build a scene: uploads the triangles, builds a bounding volume hierarchy on the
 * host and keeps it on the device.  verts_xyz [n_verts][3], tri_idx [n_tris][3]
 * (indices into verts), albedo_rgb [n_tris][3] (Lambertian, two-sided),
 * emission_rgb [n_tris][3] or NULL, lights [n_lights] with n_lights <= VRC_MAX_LIGHTS.
 * Synchronous.  Returns VRC_ERR_INVALID for bad sizes or indices, VRC_ERR_OOM. */
int vrc_build_scene(const float* verts_xyz, int32_t n_verts, const int32_t* tri_idx, int32_t n_tris,
                    const float* albedo_rgb, const float* emission_rgb, const vrc_medium* medium,
                    const vrc_point_light* lights, int32_t n_lights, vrc_scene** out);
void vrc_destroy_scene(vrc_scene* scene);

/* --------------------------------------------------------------- records */
/* Per-call record parameters.
 *   n_bands x n_bins  stratified ray set: equal d(cos theta) x equal d(phi) strata,
 *                     one jittered ray each, plus two unweighted pole rays
 *                     (Sec. 6 "Implementation": equal solid angle strata)
 *   dt                march step of the distance shells (Sec. 6)
 *   eps               error tolerance of the radius (Eq. radiusAniso3D)
 *   omega_o           outgoing direction of the phase function (unit vector)
 *   seed              jitter seed (splitmix64 counter generator)
 *   ff_signed         1: signed solid angle (closes every shell); 0: |A| as printed in App. C
 *   extrap_order      1 (Eq. radianceTaylor) or 2 (adds the Hessian term); used by the grid
 *   r_min, r_max      radius clamps
 *   rec_base          jitter index of record 0 (record i uses rec_base + i)
 *   parts             0: the whole in-scattered radiance (surface and medium shells);
 *                     1: surface shell only (the single-scattering cache of Sec. 6);
 *                     2: medium shells only (the multiple-scattering cache of Sec. 6).
 *                     With 1 or 2 every output (L, grad, hess, radius, ...) is that part.
 *   lo_grad           1: a medium vertex's outgoing radiance varies with x through the HG
 *                     phase of the light it scatters toward x (L_o(x) = L_o(x_c) f(l . w(x)) /
 *                     f(l . w(x_c)), l the light's direction of travel at the vertex, w(x) the
 *                     direction from it to x), so Eq. reducedRadianceDerivatives keeps grad L_o
 *                     and H L_o (Sec. 7 names this extension); needs exactly one light, else
 *                     VRC_ERR_UNSUPPORTED.  0 (default): L_o constant (Sec. 4). */
typedef struct {
    int32_t n_bands, n_bins;
    float dt, eps;
    float omega_o[3];
    uint64_t seed;
    int32_t ff_signed;
    int32_t extrap_order;
    float r_min, r_max;
    int64_t rec_base;
    int32_t parts;
    int32_t lo_grad;
} vrc_record_params;

/* Caller-allocated device outputs of vrc_compute_records, one row per record.
 * Required: L, grad, hess, radius, status, pos.  Others may be NULL.
 *   L [n][3]        Monte Carlo in-scattered radiance (Eq. outLF, Sec. 4 last paragraph)
 *   grad [n][9]     occlusion-aware gradient (Eq. SegmentRadianceGradient)
 *   hess [n][18]    occlusion-aware Hessian (Eq. SegmentRadianceHessian)
 *   *_ss / *_ms     the same split into surface-shell (single scattering, surface
 *                   radiance) and medium-shell (second bounce) parts
 *   L_ff [n][3]     triangulated radiance of Eq. ApprxRadiance (diagnostic)
 *   radius [n]      validity radius (Eq. radiusAniso3D with the largest |eigenvalue|)
 *   eig [n][3]      eigenvalues of the luminance Hessian, ascending
 *   kappa [n]       sum of per-cell Hessian norms / norm of their sum (conditioning)
 *   status [n]      VRC_REC_* bits
 *   pos [n][3]      the record centres (copied from d_pos)
 *   n_cells [n]     cells evaluated (lit cells of all shells; work counter), NULL to skip
 *   n_far [n]       furthest-vertex evaluations (sum of tie sizes over lit cells), NULL to skip
 *   n_shells [n]    medium shells K = ceil(max t_end / dt), NULL to skip
 *   log_radius [n]  natural log of the radius (training target of the learned predictor), NULL to skip
 *   hit_prim, hit_t [n][dbg_stride]  per-ray primary hit id (-1 = escaped) and t,
 *                   for rays v < n_bands*n_bins + 2; NULL to skip
 *   radii [n][3]    ellipsoidal record (Eq. radiusAniso3D per eigenvalue, Sec. 5): the
 *                   principal radius along each eigenvector of the luminance Hessian, in
 *                   the order of eig, clamped to [r_min, r_max]; NULL to skip
 *   axes [n][9]     the matching unit eigenvectors, row i for eig[i] (FP64 solve, stored
 *                   as float); NULL to skip.  Eigenvectors of equal eigenvalues are any
 *                   orthonormal basis of their eigenspace (the ellipsoid is unique).
 *   dbg_lit [n][dbg_shells][(dbg_stride + 31) / 32]  (debug, NULL to skip; needs hit_prim)
 *                   bit v of row k is set when vertex v of shell k (k = 0 the surface
 *                   shell, k >= 1 medium shell k; rays in hit_prim's order) has nonzero
 *                   radiance: the record's visibility decisions.  The caller zeroes the
 *                   buffer; shells k >= dbg_shells are not written. */
typedef struct {
    float* L;
    float* grad;
    float* hess;
    float* L_ss;
    float* grad_ss;
    float* hess_ss;
    float* L_ms;
    float* grad_ms;
    float* hess_ms;
    float* L_ff;
    float* radius;
    float* eig;
    float* kappa;
    int32_t* status;
    float* pos;
    int32_t* n_cells;
    int32_t* n_far;
    int32_t* n_shells;
    float* log_radius;
    int32_t* hit_prim;
    float* hit_t;
    int32_t dbg_stride;
    float* radii;
    float* axes;
    uint32_t* dbg_lit;
    int32_t dbg_shells;
} vrc_records_view;

/* Launch shape of the record kernel (see vrc_autotune_records). 0 = library default: for at
 * most one record per SM, 512 threads with the whole ray set (up to 200 KB); for small ray
 * sets (whole set within 36 KB) and at least 6 records per SM, 128 threads with the whole ray
 * set (six blocks per SM); else 384 threads with the whole ray set in shared memory when that
 * fits two blocks per SM (up to 110 KB); else 256 threads with as many bands per chunk as fit
 * 72 KB (three blocks). */
typedef struct {
    int32_t threads;        /* threads per block: 128, 256, 384, 512 */
    int32_t chunk_bands;    /* bands of the ray set kept in shared memory at once */
    int32_t blocks_per_sm;  /* persistent blocks per SM */
    int32_t shadow_bvh;     /* 1: shadow rays traverse the BVH; 0: light buffer (default) */
    int32_t no_prepass;     /* 1: the record kernel traces its primary rays itself; 0 (default):
                               uniform ray sets of up to 64 Mi rays per call are traced first by
                               a flat pre-pass kernel into scene-owned buffers (28 B per ray) */
} vrc_record_tuning;

/* Compute n records at d_pos [n][3] (Secs. 4-5 and App. A, C): trace the stratified
 * ray set through the scene, build the distance shells (zero-radiance samples at
 * occluders), evaluate every cell's form factor, transmittance and phase terms with
 * their derivatives, reduce them into L, grad L and H L, and set each radius from the
 * Hessian's eigenvalues.  d_n_bands [n] (nullable) gives per-record band counts with
 * bins = 2 * bands (mixed ray counts in one persistent launch); each must lie in
 * [2, params->n_bands] (shared memory is sized for params->n_bands), a record outside
 * that range gets zero outputs and status VRC_REC_BAD_COUNT.  Asynchronous on
 * `stream`.  The radius stage (luminance eigen-solve, Eq. radiusAniso3D) runs as a
 * second kernel on the same stream.  VRC_ERR_INVALID for null required outputs, n < 0,
 * bands < 1, bins < 3, parts outside 0..2; VRC_ERR_UNSUPPORTED for more than 256 bands
 * or 512 bins. */
int vrc_compute_records(vrc_scene* scene, const float* d_pos, int32_t n, const int32_t* d_n_bands,
                        const vrc_record_params* params, const vrc_records_view* d_out, void* stream);

/* Same computation from HOST buffers: h_pos [n][3] in, h_L [n][3], h_grad [n][9],
 * h_hess [n][18], h_radius [n], h_status [n] out (any output may be NULL).  Copies
 * in and out through device buffers owned by the scene; synchronous. */
int vrc_compute_records_host(vrc_scene* scene, const float* h_pos, int32_t n, const vrc_record_params* params,
                             float* h_L, float* h_grad, float* h_hess, float* h_radius, int32_t* h_status);

/* One whole step of the cache from HOST buffers (Secs. 4-6: records, then queries by
 * Eq. radianceTaylor): h_pos [n][3] in -> records as vrc_compute_records (parts and
 * extrap_order from params) -> the record grid -> nq queries h_q [nq][3] -> h_rgb [nq][3]
 * and h_qstatus [nq] (as vrc_query_inscatter), and the records h_L [n][3], h_grad [n][9],
 * h_hess [n][18], h_radius [n], h_status [n] (each may be NULL).  *grid: NULL on the first
 * call, which builds the grid and stores it there (the caller frees it with
 * vrc_destroy_grid); later calls rebuild it in place.  The copies run in device buffers
 * and on two streams owned by the scene: the queries are uploaded while the records are
 * computed, the records downloaded while the grid and the queries run; host buffers must
 * be page-locked for the copies to overlap.  Synchronous: every output is in host memory
 * on return.  VRC_ERR_INVALID for bad sizes or null buffers, else as the calls it makes. */
int vrc_cache_step_host(vrc_scene* scene, vrc_grid** grid, const float* h_pos, int32_t n,
                        const vrc_record_params* params, const float* h_q, int32_t nq, float* h_L, float* h_grad,
                        float* h_hess, float* h_radius, int32_t* h_status, float* h_rgb, int32_t* h_qstatus);

int vrc_set_record_tuning(vrc_scene* scene, const vrc_record_tuning* tuning);
int vrc_get_record_tuning(const vrc_scene* scene, vrc_record_tuning* tuning);

/* Per-kernel timing of vrc_compute_records (no counterpart in the paper; measurement).
 * vrc_record_timing(scene, 1) starts recording CUDA events on the launching stream around
 * the three kernels of each call (primary pre-pass, record kernel, radius stage) -- at most
 * 64 calls, none while the stream is captured into a graph; 0 stops.  vrc_record_kernel_times
 * waits for the recorded events, writes the summed milliseconds of the three kernels to
 * ms3[3] and the number of timed calls to *launches, and clears the record. */
int vrc_record_timing(vrc_scene* scene, int32_t enable);
int vrc_record_kernel_times(vrc_scene* scene, float* ms3, int32_t* launches);

/* Autotuner for the record kernel's launch shape (threads per block, bands per chunk and,
 * for uniform ray sets, the primary pre-pass on or off).
 * Times each candidate on up to 16,384 of the given records (one warm-up launch and two
 * timed launches each, CUDA events on `stream`), keeps the fastest in the scene, writes
 * it to *best and caches it per (bands, bins, mixed-count flag, parts, log2 of n, log2
 * of the scene's triangle count).  A cached
 * entry is reused without timing.  d_out is overwritten by the trial launches (its final
 * contents are a correct evaluation of the first records).  Synchronous. */
int vrc_autotune_records(vrc_scene* scene, const float* d_pos, int32_t n, const int32_t* d_n_bands,
                         const vrc_record_params* params, const vrc_records_view* d_out, void* stream,
                         vrc_record_tuning* best);

/* CUDA graph of one vrc_compute_records call (work-counter reset, largest-first ordering
 * for mixed ray counts, the persistent record kernel) with fixed buffers: replaying it
 * recomputes the records from the current contents of d_pos / d_n_bands into d_out.
 * The scene's current tuning is baked in.  Create is synchronous; launch is asynchronous
 * on `stream`; the graph must be destroyed before the scene. */
typedef struct vrc_graph vrc_graph;
int vrc_records_graph_create(vrc_scene* scene, const float* d_pos, int32_t n, const int32_t* d_n_bands,
                             const vrc_record_params* params, const vrc_records_view* d_out, vrc_graph** out);
int vrc_graph_launch(vrc_graph* graph, void* stream);
void vrc_graph_destroy(vrc_graph* graph);

/* --------------------------------------------------------------- queries */

/* Build the lookup structure for Eq. radianceTaylor from n device records (pos,
 * radius, L, grad and, for extrap_order 2, hess of `recs`): a compact record table
 * and a uniform grid over the unit cube whose cells list every record whose sphere
 * of radius R_k overlaps them.  The grid owns copies; `recs` may be freed after the
 * call completes on `stream`.  Synchronous (reads back the list size). */
int vrc_build_record_grid(const vrc_records_view* recs, int32_t n, int32_t extrap_order, vrc_grid** out,
                          void* stream);
void vrc_destroy_grid(vrc_grid* grid);

/* The same structure for ellipsoidal records (Eq. radiusAniso3D per eigenvalue, Sec. 5;
 * anisotropic cache points, Sec. 6): record k covers the points with D^T M_k D < 1,
 * D = x' - x_k, M_k = sum_i v_i v_i^T / R_i^2 from `radii` and `axes` of `recs` (both
 * required), and vrc_query_inscatter on this grid uses rho = sqrt(D^T M_k D) in place of
 * |D| / R_k (membership rho < 1, d = 1 - rho).  Cells list every record whose bounding
 * box and bounding sphere (largest radius) both meet them.  Same ownership, errors and
 * synchronisation as vrc_build_record_grid. */
int vrc_build_record_grid_aniso(const vrc_records_view* recs, int32_t n, int32_t extrap_order, vrc_grid** out,
                                void* stream);

/* Rebuild `grid` in place from n records (spheres, or ellipsoids with aniso = 1), as
 * vrc_build_record_grid(_aniso) would build it, reusing the grid's device buffers where
 * they are large enough (growing them otherwise).  Same requirements, errors and
 * synchronisation; on an error the grid may only be destroyed or rebuilt. */
int vrc_rebuild_record_grid(vrc_grid* grid, const vrc_records_view* recs, int32_t n, int32_t extrap_order,
                            int32_t aniso, void* stream);

/* Answer nq queries d_q [nq][3] by Eq. radianceTaylor: the weighted first-order (or,
 * with extrap_order 2, second-order) Taylor extrapolation from every record k with
 * |x' - x_k| < R_k, weight w = 3d^2 - 2d^3, d = 1 - |x' - x_k| / R_k.  Writes d_rgb
 * [nq][3] and d_status [nq] = number of contributing records (0 = miss, rgb = 0).
 * Asynchronous on `stream`. */
int vrc_query_inscatter(const vrc_grid* grid, const float* d_q, int32_t nq, float* d_rgb, int32_t* d_status,
                        void* stream);

/* --------------------------------------------------------------- 2D world
 * The paper's two-dimensional world (Sec. 3; Sec. 4 in 2D; App. A; App. B; Eq.
 * radiusAniso2D): light travels, scatters and is absorbed in the plane, radiance from a
 * point source falls off as 1/r, the isotropic phase function is 1/(2 pi).  Geometry is
 * a set of line segments (two-sided Lambertian curves, BRDF albedo / 2) in the unit
 * square, which the homogeneous medium fills. */
typedef struct { float pos[2]; float intensity[3]; } vrc2d_point_light;
typedef struct vrc2d_scene vrc2d_scene;

/* Upload a 2D scene: segs [n][4] (x0, y0, x1, y1), albedo [n][3] (host arrays, copied);
 * sigma_s, sigma_a of the medium; up to VRC_MAX_LIGHTS point lights.  VRC_ERR_INVALID for
 * a zero-length segment or bad sizes.  Synchronous. */
int vrc2d_build_scene(const float* segs, int32_t n_segs, const float* albedo, float sigma_s, float sigma_a,
                      const vrc2d_point_light* lights, int32_t n_lights, vrc2d_scene** out);
void vrc2d_destroy_scene(vrc2d_scene* scene);

/* n 2D records at d_pos [n][2] (device): N = params->n_bins equal-angle strata with one
 * jittered ray each (params->n_bands must be 1), distance shells every params->dt, every
 * shell's cells (segments between angularly adjacent vertices) with App. B's angle
 * derivatives and App. A's transmittance derivatives, the radius of Eq. radiusAniso2D.
 * Results go to `out` in the 3D layout of vrc_records_view, in the plane z = 0.5: pos
 * (x, y, 0.5), grad [c] = (d/dx, d/dy, 0), hess [c] = (xx, xy, 0, yy, 0, 0), eig = the
 * 2D eigenvalues and 0 in ascending order, radii / axes = the ellipse's principal radii
 * (Eq. radiusAniso2D per eigenvalue) with the plane's normal as third axis (radius
 * r_max), so vrc_build_record_grid(_aniso) and vrc_query_inscatter answer 2D queries at
 * z = 0.5.  params->parts selects surface shell / medium shells as for 3D records.
 * out->hit_prim / hit_t (debug, nullable) receive each ray's hit segment (-1 = none) and
 * t at [rec][ray], dbg_stride >= N.  Asynchronous on `stream`.  VRC_ERR_INVALID for bad
 * parameters; VRC_ERR_UNSUPPORTED for more than 4096 directions. */
int vrc2d_compute_records(vrc2d_scene* scene, const float* d_pos, int32_t n, const vrc_record_params* params,
                          const vrc_records_view* out, void* stream);

/* --------------------------------------------------------------- renderer
 * The renderer around the cache (Sec. 6): camera rays marched through the medium with the
 * paper's uniform ray marching, cache look-ups at the march points, adaptive placement.
 * Camera: pinhole at pos looking along forward (up = +z), vertical field of view in
 * degrees, width x height pixels.  A pixel's ray is marched from its entry into the unit
 * cube to min(first hit, cube exit) in `steps` equal segments; the march points are the
 * segment midpoints; a pixel's value is sum_k ds sigma_s exp(-sigma_t s_k) L(x_k). */
typedef struct { float pos[3]; float forward[3]; float vfov_deg; int32_t width, height; } vrc_camera;

/* March points of the pixels (x0 + i*stride, y0 + j*stride), i < w, j < h: d_pts
 * [w*h*steps][3] (pixel-major, then step), d_valid [w*h*steps] (0 where the pixel's ray
 * misses the medium).  Asynchronous. */
int vrc_march_points(vrc_scene* scene, const vrc_camera* cam, int32_t x0, int32_t y0, int32_t w, int32_t h,
                     int32_t stride, int32_t steps, float* d_pts, int32_t* d_valid, void* stream);

/* Render the w x h pixel rectangle at (x0, y0) from an order-1 grid: d_img [w*h][3]; d_miss
 * [w*h] (nullable) = march points of the pixel that no record covers (they contribute 0).
 * grid2 (nullable): a second order-1 grid whose look-up is added to the first -- the
 * separate single- and multiple-scattering caches of Sec. 6 (records computed with
 * parts 1 and 2); a march point then counts once in d_miss per cache that misses it.
 * Asynchronous. */
int vrc_render(vrc_scene* scene, const vrc_grid* grid, const vrc_grid* grid2, const vrc_camera* cam, int32_t x0,
               int32_t y0, int32_t w, int32_t h, int32_t steps, float* d_img, int32_t* d_miss, void* stream);

/* The same for a list of pixels (linear index y * width + x): march points [n_pix*steps][3]
 * in list order; render writes each listed pixel at its own index of the full-frame
 * d_img [width*height][3] / d_miss.  Asynchronous. */
int vrc_march_pixels(vrc_scene* scene, const vrc_camera* cam, const int32_t* d_pix, int32_t n_pix, int32_t steps,
                     float* d_pts, int32_t* d_valid, void* stream);
int vrc_render_pixels(vrc_scene* scene, const vrc_grid* grid, const vrc_grid* grid2, const vrc_camera* cam,
                      const int32_t* d_pix, int32_t n_pix, int32_t steps, float* d_img, int32_t* d_miss, void* stream);

/* Indices i (ascending) with d_flags[i] != 0 into d_idx; their number to *h_count
 * (synchronous).  d_scratch holds 2 n + n/1024 + 2 ints. */
int vrc_compact_indices(const int32_t* d_flags, int32_t n, int32_t* d_scratch, int64_t scratch_ints, int32_t* d_idx,
                        int32_t* h_count, void* stream);

/* Pixel values from caller-given radiance at every march point (d_L [w*h*steps][3], in
 * vrc_march_points order) -- e.g. a full record at every point, the reference image. */
int vrc_composite(vrc_scene* scene, const vrc_camera* cam, int32_t x0, int32_t y0, int32_t w, int32_t h,
                  int32_t steps, const float* d_L, float* d_img, void* stream);

/* Placement wave (Sec. 6: a record is added where no valid record exists): among the
 * candidates with 0 <= d_level[i] <= level, pick in each cell of a 2^level grid over the
 * cube the one with the smallest index.  Writes the picked indices (ascending) and their
 * positions to d_site_idx / d_site_pts and their number to *h_count, and (h_pool non-NULL)
 * the number of candidates still in the pool at any level (d_level[i] >= 0) to *h_pool, so
 * that a caller can end its waves once the pool is empty (synchronous).
 * d_scratch must hold 8^level + 2 n + n/1024 + 3 ints; level <= 8. */
int vrc_select_sites(const float* d_pts, const int32_t* d_level, int32_t n, int32_t level, int32_t* d_scratch,
                     int64_t scratch_ints, int32_t* d_site_idx, float* d_site_pts, int32_t* h_count,
                     int32_t* h_pool, void* stream);

/* Placement wave over several levels at once (learned placement, not in the paper): every
 * candidate with lmin <= d_level[i] <= lmax competes in its cell of the 2^d_level[i] grid,
 * and the candidate with the smallest index in each (level, cell) is picked, so that one
 * wave places the sites of every level.  Outputs as vrc_select_sites (*h_count sites, in
 * ascending candidate order; *h_pool, when non-NULL, the candidates left in the pool at any
 * level); synchronous.  lmax <= 7; d_scratch must hold (8^(lmax+1) - 8^lmin)/7 + 2 n +
 * n/1024 + 3 ints. */
int vrc_select_sites_levels(const float* d_pts, const int32_t* d_level, int32_t n, int32_t lmin, int32_t lmax,
                            int32_t* d_scratch, int64_t scratch_ints, int32_t* d_site_idx, float* d_site_pts,
                            int32_t* h_count, int32_t* h_pool, void* stream);

/* d_level[i] = min(d_level[i] + 1, lmax) for the candidates still in the pool (d_level[i] >=
 * 0): after a wave, the uncovered candidates compete on the next finer grid.  Asynchronous. */
int vrc_bump_levels(int32_t* d_level, int32_t n, int32_t lmax, void* stream);

/* Learned levels predicted once per cell: after vrc_select_sites at cell_level (which left
 * each cell's representative -- smallest candidate index -- in the first 8^cell_level
 * ints of d_scratch), d_site_logr[j] is the predicted log radius of site j (index
 * d_site_idx[j]); every pool candidate takes its cell representative's level
 * (as in vrc_levels_from_radius).  d_rep_level [n] is scratch.  Asynchronous. */
int vrc_levels_by_cell(const float* d_pts, int32_t n, int32_t cell_level, const int32_t* d_scratch,
                       const int32_t* d_site_idx, const float* d_site_logr, int32_t n_sites, float cell_over_radius,
                       int32_t lmin, int32_t lmax, int32_t* d_rep_level, int32_t* d_level, void* stream);

/* d_level[i] = start_level where d_valid[i] != 0, else -1 (not a candidate).  Asynchronous. */
int vrc_init_levels(const int32_t* d_valid, int32_t n, int32_t start_level, int32_t* d_level, void* stream);

/* d_level[i] = -1 (leaves the candidate pool) where d_count[i] > 0.  Asynchronous. */
int vrc_update_coverage(const int32_t* d_count, int32_t n, int32_t* d_level, void* stream);

/* d_level[i] = -1 where d_level[i] == level: the candidates of one level leave a (copy of
 * the) pool, so that site selection level by level picks each candidate at its own level
 * only (one-shot placement).  Asynchronous. */
int vrc_retire_level(int32_t* d_level, int32_t n, int32_t level, void* stream);

/* Fallback rule of the learned radius (not in the paper): the predicted radius R^ =
 * exp(d_logr[i] + logr_offset) (the offset carries a prediction made at the training
 * tolerance eps0 to eps: R goes as eps^(1/5) by Eq. radiusAniso3D, so the offset is
 * log(eps / eps0) / 5) is kept only where a record of the coarse ray set at the same
 * point says its error is within the tolerance -- the error at R of Eq. radiusAniso3D,
 * 4 pi |lambda| R^5 / (15 L), is at most eps exactly when R is at most that coarse
 * record's radius d_radius_coarse[i] (computed at eps).  Elsewhere d_logr_out[i] =
 * logr_fallback (a caller's value that sends the candidate to plain placement) and
 * *d_n_fallback (device, caller-zeroed) is incremented.  d_radius_coarse NULL: the offset
 * only.  Asynchronous. */
int vrc_mlp_fallback(const float* d_logr, int32_t n, float logr_offset, const float* d_radius_coarse,
                     float logr_fallback, float* d_logr_out, int32_t* d_n_fallback, void* stream);

/* Learned placement level of each pool candidate from a predicted log radius: the finest
 * level whose cell is at most cell_over_radius x the predicted radius, in [lmin, lmax]. */
int vrc_levels_from_radius(const float* d_logr, int32_t n, float cell_over_radius, int32_t lmin, int32_t lmax,
                           int32_t* d_level, void* stream);

/* --------------------------------------------------------------- learned radius
 * Not in the paper: a small network predicts a record's log validity radius from a cheap
 * coarse ray set, so full records are computed only where they are needed; the full
 * record decides (its radius sets coverage).
 *
 * vrc_coarse_features: for each position d_pos[i], the coarse stratified ray set of
 * `params` (n_bands x n_bins, jitter seed, rec_base; pole rays excluded) gives
 * d_feat[i][v] = log(distance to the first hit or the cube exit) and
 * d_feat[i][N + v] = sum over lights of transmittance x visibility from that point,
 * N = n_bands * n_bins (N = 128 for the network's 256 inputs).  Asynchronous. */
int vrc_coarse_features(vrc_scene* scene, const float* d_pos, int32_t n, const vrc_record_params* params,
                        float* d_feat, void* stream);
/* The same features as BF16 (round to nearest even), 512 B per record: the input of
 * vrc_mlp_predict_bf16.  d_feat [n][2 N] BF16, 16-byte aligned.  Asynchronous. */
int vrc_coarse_features_bf16(vrc_scene* scene, const float* d_pos, int32_t n, const vrc_record_params* params,
                             void* d_feat, void* stream);

/* The network: 256 -> 64 -> GELU -> 64 -> GELU -> 1 (log radius), BF16 weights and
 * activations as tensor-core operands, FP32 accumulation.  Parameters are one float
 * vector of vrc_mlp_num_params() = 20,673 values: W1 [64][256], b1 [64], W2 [64][64],
 * b2 [64], w3 [64], b3 [1]; the library keeps an FP32 master copy and AdamW moments.
 * create copies the initial parameters (host, required: the caller draws them);
 * get/set copy parameters, moments and step count (checkpoint and resume; moments may be
 * NULL).  predict: d_logr[n] from d_feat[n][256] (16-byte aligned).  gradient: the MSE
 * loss gradient over the n examples into d_grad (NULL: internal buffer) and, optionally,
 * the predictions into d_pred.  train_step: gradient + one AdamW step (betas 0.9, 0.999,
 * eps 1e-8, decoupled weight decay); *h_loss (nullable, then synchronous) = mean squared
 * residual before the step.  status reports VRC_ERR_TIMEOUT if a bounded device wait of a
 * tensor-core kernel gave up. */
typedef struct vrc_mlp vrc_mlp;
int vrc_mlp_create(const float* h_params, vrc_mlp** out);
void vrc_mlp_destroy(vrc_mlp* mlp);
int32_t vrc_mlp_num_params(void);
int vrc_mlp_get_params(const vrc_mlp* mlp, float* h_params, float* h_adam_m, float* h_adam_v, int64_t* h_step);
int vrc_mlp_set_params(vrc_mlp* mlp, const float* h_params, const float* h_adam_m, const float* h_adam_v,
                       int64_t step);
int vrc_mlp_predict(const vrc_mlp* mlp, const float* d_feat, int32_t n, float* d_logr, void* stream);
/* vrc_mlp_predict from BF16 features d_feat [n][256] (row-major, 16-byte aligned): each
 * 128-row tile is copied from HBM into the tensor cores' operand layout by the tensor
 * memory accelerator (tiled bulk copies, 128-byte swizzle), half the bytes of the FP32
 * path; the result equals vrc_mlp_predict on the same features rounded to BF16.
 * VRC_ERR_UNSUPPORTED when the CUDA driver offers no tensor-map encoder.  Asynchronous. */
int vrc_mlp_predict_bf16(const vrc_mlp* mlp, const void* d_feat, int32_t n, float* d_logr, void* stream);
int vrc_mlp_gradient(vrc_mlp* mlp, const float* d_feat, const float* d_target, int32_t n, float* d_grad,
                     float* d_pred, void* stream);
int vrc_mlp_train_step(vrc_mlp* mlp, const float* d_feat, const float* d_target, int32_t n, float lr,
                       float weight_decay, float* h_loss, void* stream);
int vrc_mlp_status(const vrc_mlp* mlp);

/* Queries for callers that cannot allocate device memory.
 *
 * No counterpart in the paper: this is a library convenience.  vrc_query_inscatter
 * needs a vrc_grid, which vrc_build_record_grid allocates; some callers cannot call
 * cudaMalloc at query time -- a host application or plugin framework that owns all
 * device memory and hands out fixed pools, a real-time renderer that forbids
 * allocation after start-up because cudaMalloc may synchronise the device and stall
 * its other streams, a service with a hard pre-reserved memory budget.  This entry
 * point answers the same queries as a grid of sphere records from vrc_build_record_grid
 * (same Eq. radianceTaylor, same results within float rounding) straight from the
 * caller's record buffers and allocates nothing: no cudaMalloc, cudaFree or allocating
 * library routine.  Ellipsoidal regions are not served: the radii and axes fields are
 * ignored and each record's sphere of radius R_k is used.  Its working memory is one
 * file-scope device array of VRC_NOALLOC_SCRATCH_INTS 32-bit words (4 MiB).
 *   recs     device records: pos, radius, L, grad (and hess for extrap_order 2)
 *   n        number of records, at most VRC_NOALLOC_MAX_RECORDS (else VRC_ERR_UNSUPPORTED)
 *   d_q, nq, d_rgb, d_status   as for vrc_query_inscatter
 * The first call on a device looks up the array's device address (cudaGetSymbolAddress)
 * with that device current.  CUDA loads a library's device code lazily by default, so
 * that first call may also load the module and reserve the array on the device, which
 * can synchronise the device or fail (VRC_ERR_CUDA) when memory is short: make the first
 * call during start-up, before any stream capture.  From then on the device holds the
 * array until the process exits.  Every
 * call reuses the same array and leaves its contents behind, so two calls that overlap
 * on the GPU (different streams without ordering, or concurrent host threads) race and
 * may return wrong results: order them on one stream.  If the record lists do not fit
 * in the array the queries scan every record instead (same answer, slower).
 * Asynchronous on `stream`. */
#define VRC_NOALLOC_SCRATCH_INTS (1 << 20)
#define VRC_NOALLOC_MAX_RECORDS 65536
int vrc_query_inscatter_noalloc(const vrc_records_view* recs, int32_t n, int32_t extrap_order, const float* d_q,
                                int32_t nq, float* d_rgb, int32_t* d_status, void* stream);

/* --------------------------------------------------------------- misc */
const char* vrc_status_string(int status);
int vrc_version(void);

#ifdef __cplusplus
}
#endif
#endif /* VRC_H */
