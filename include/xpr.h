/*
 * xpr.h -- C ABI of the GB300 (sm_103a) 3D Gaussian Splatting tile-splatting
 * library (libxpr.so).
 *
 * The path follows the four-stage point-based pipeline of arXiv 2606.11529
 * (Sec. 2 and Sec. 4): Preprocess (project each primitive), Rasterizer
 * (replicate each primitive over the tiles of its bounding box, assign tile
 * IDs, cull, sort by (tile, depth), find per-tile segment bounds) and Shader
 * (front-to-back alpha compositing per pixel), plus the reverse-order adjoint
 * of the shader and of the projection.  The 3DGS instance of the per-element
 * functions is the paper's Listing 1 (project, tile_cull, evaluate).
 *
 * Conventions for every entry point
 *   - All array pointers are DEVICE pointers (CUDA global memory) unless the
 *     comment says "host".  The caller allocates and owns every buffer; the
 *     library never allocates device memory and keeps no state between calls
 *     except a per-host-thread last-error string, a process-wide counter of
 *     launched kernels and, per host thread and device, a 64-byte page-locked
 *     host buffer with two events for the counts the binning by rows reads
 *     back.
 *   - `stream` is a cudaStream_t (NULL = legacy default stream).  Work is
 *     enqueued asynchronously on it; entry points that must return a count to
 *     the host (xpr_tile_bin, xpr_bin_sorted, xpr_bin_rows) synchronise that
 *     stream.
 *   - Floating-point arrays are IEEE float32, row-major, densely packed.
 *   - Return value: an XprStatus.  On error nothing is guaranteed about the
 *     output buffers; xpr_last_error() describes the failure.
 *   - Sizes: primitive count n < 2^31, intersection count < 2^31, image
 *     width and height in [1, 32768], tile sizes 8 or 16.
 */
#ifndef XPR_H
#define XPR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum XprStatus {
    XPR_OK = 0,
    XPR_ERR_INVALID = 1,  /* bad argument: NULL pointer, size out of range, unsupported tile size */
    XPR_ERR_CAPACITY = 2, /* intersection buffer too small; the required count is reported */
    XPR_ERR_CUDA = 3,     /* a CUDA launch or runtime call failed */
    XPR_ERR_TIMEOUT = 4,  /* a bounded device-side wait expired */
    XPR_ERR_INTERNAL = 5  /* a device-side consistency check failed */
} XprStatus;

/* Pinhole camera (the paper's `cam` and `view` arguments of project, Sec. 3.1).
 * viewmat: world-to-camera [R | t], 3x4 row-major; camera axes x right,
 * y down, z forward.  Pixel (x, y) of a 3DGS image is evaluated at the raw
 * coordinate (x, y) as in Listing 1 evaluate. */
typedef struct XprCamera {
    int32_t width, height;
    float fx, fy, cx, cy;
    float viewmat[12];
    float z_near; /* primitives with camera-space z <= z_near are invisible (Listing 1 visibility flag) */
    int32_t model; /* 0 = pinhole; 1 = fisheye (3DGUT configs only): a camera-space point at angle
                      theta = atan2(sqrt(x^2 + y^2), z) from the axis lands at (fx theta_d x / r + cx,
                      fy theta_d y / r + cy), theta_d = theta (1 + k1 theta^2 + k2 theta^4 + k3 theta^6
                      + k4 theta^8), r = sqrt(x^2 + y^2) */
    float dist[4]; /* fisheye k1..k4 (ignored for the pinhole) */
} XprCamera;

/* Renderer constants.  alpha_thresh is the contribution threshold 1/255 of
 * the Appendix (3DGS implementation); alpha_max (0.99), t_eps (1e-4),
 * cov_dilation (0.3) and clip_factor (1.3, limit on |x/z| relative to the
 * half field of view inside the EWA Jacobian) are the 3DGS conventions the
 * paper's compute_cov_2D / blend loop leave to the config. */
typedef struct XprConfig {
    int32_t tile_w, tile_h; /* 8 or 16 each (the paper's GPU tile sizes, hyperparameter table) */
    float alpha_thresh;
    float alpha_max;
    float t_eps;        /* stop when T (1 - alpha) < t_eps, before blending that primitive */
    float cov_dilation;
    float clip_factor;
    int32_t sh_degree;  /* 0..3; K = (sh_degree + 1)^2 coefficients per colour channel */
    float bg[3];        /* background colour added as T_final * bg */
    int32_t batch_depth;/* render: entries staged per shared-memory batch; 0 = kernel default */
    int32_t method;     /* XPR_METHOD_3DGS (0), XPR_METHOD_3DGUT (1) or XPR_METHOD_LINPRIM (2): selects
                           the binning's tile cull (3DGUT: ray-offset bounds; LinPrim: the chord bound
                           of xpr_tile_bin_lp) and which projection / render entry points accept the
                           config (each refuses the other methods) */
} XprConfig;

#define XPR_METHOD_3DGS 0
#define XPR_METHOD_3DGUT 1
#define XPR_METHOD_LINPRIM 2

/* 3DGS PrimitiveParams (Appendix, 3DGS implementation), structure of arrays:
 * mu[n,3] world-space means, scale[n,3] (positive, activated), quat[n,4]
 * rotation (w, x, y, z; normalised inside), opacity[n] (activated, in (0,1)),
 * sh[n,K,3] spherical-harmonic coefficients (real SH, Condon-Shortley
 * phase; colour = max(0, sum_k sh_k Y_k(d) + 0.5), d = unit vector from the
 * camera centre to mu). */
typedef struct XprPrims {
    const float *mu;
    const float *scale;
    const float *quat;
    const float *opacity;
    const float *sh;
} XprPrims;

/* Gradients with the same layout as XprPrims. */
typedef struct XprPrimsGrad {
    float *mu;
    float *scale;
    float *quat;
    float *opacity;
    float *sh;
} XprPrimsGrad;

/* Projected record, 12 floats per primitive (the paper's shader data p_sd,
 * tile-cull data p_tcd and depth of ProjectResult, Listing 1):
 *   [0] mu_2D.x  [1] mu_2D.y  [2] conic00  [3] conic01  [4] conic11
 *   [5] opacity  [6] r  [7] g  [8] b  [9] depth (camera z)
 *   [10] ln(opacity / alpha_thresh)  [11] visible (1.0 or 0.0)
 * conic = Sigma_2D^{-1}.  Invisible primitives have every entry 0 except
 * depth.  The same layout is used for screen-space gradients (d_rec):
 *   [0..1] d mu_2D, [2..4] d conic, [5] d opacity, [6..8] d rgb, [9] d depth
 *   (nonzero only from rendered depth, xpr_render_bwd_feat), rest 0. */
#define XPR_REC_FLOATS 12

/* One item of a multi-scene launch: a scene (a range of primitives of the
 * concatenated parameter arrays) seen by one camera.  Items are listed in
 * order; every offset is the previous item's plus its size:
 *   prim_offset, n: the scene's primitives [prim_offset, prim_offset + n) of
 *     the concatenated XprPrims arrays (several items may name one scene);
 *   rec_offset: the item's first record; records are item-major and each
 *     item's block is padded to a multiple of 32 records (item k + 1 starts at
 *     rec_offset + ceil(n / 32) 32), the padding records being invisible;
 *   tile_offset: the item's first global tile id (item k + 1 starts at
 *     tile_offset + tiles_x tiles_y of item k's camera);
 *   pix_offset: the item's first pixel in the per-pixel buffers (t_final,
 *     n_contrib: pix_offset + W H of the next; image planes [3, H, W] at
 *     3 pix_offset floats). */
typedef struct XprItem {
    int64_t prim_offset;
    int64_t n;
    int64_t rec_offset;
    int64_t tile_offset;
    int64_t pix_offset;
} XprItem;

/* ---- Preprocess ----------------------------------------------------------
 * xpr_project: Listing 1 project for n primitives (Sec. 4.1 Preprocess):
 * camera-space mean, Sigma = R S S^T R^T, EWA footprint Sigma_2D = J W Sigma
 * W^T J^T + dilation I, conic, opacity-aware extents sqrt(2 ln(o/a_t)
 * Sigma_2D,xx) (and yy), half-open tile bounding box, tile count, visibility
 * flag (det > 0, o >= a_t, r > 0, tc > 0, z > z_near) and SH colour.
 * Outputs: rec[n,12], bbox[n,4] int32 (xmin, ymin, xmax, ymax in tiles,
 * half-open; zero when invisible), tile_count[n] int32 (bounding-box tile
 * count tc of Sec. 4.2; 0 when invisible).  isect_count[n] int32 (may be
 * NULL): number of tiles of the box that pass the tile cull of xpr_tile_bin,
 * i.e. the exact number of pairs the primitive will emit (the binning then
 * needs no counting pass of its own).  prims->sh may be NULL: the records'
 * colours are then left 0 and xpr_project_color fills them later (binning and
 * sorting read only the geometry, so the SH coefficients can still be on
 * their way to the device while those stages run). */
int xpr_project(const XprPrims *prims, int64_t n, const XprCamera *cam, const XprConfig *cfg, float *rec,
                int32_t *bbox, int32_t *tile_count, int32_t *isect_count, void *stream);

/* xpr_project_host: xpr_project whose geometry (mu, scale, quat, opacity) is
 * read straight from page-locked host memory (`host`: pointers of pinned
 * allocations, which the device addresses through the host link), and which
 * writes a copy of that geometry into the device arrays of `dst` in the same
 * pass (later passes, e.g. xpr_project_bwd, read dst).  The projection then
 * runs at the host link's bandwidth instead of after a separate copy.
 * host->sh is ignored; dst->sh is a DEVICE pointer or NULL (colours left for
 * xpr_project_color, as in xpr_project).  Every host pointer must lie in
 * page-locked memory mapped for the device: otherwise XPR_ERR_INVALID and
 * nothing is launched.  dst->quat, rec and bbox 16-byte aligned.  Outputs as
 * xpr_project. */
int xpr_project_host(const XprPrims *host, const XprPrims *dst, int64_t n, const XprCamera *cam,
                     const XprConfig *cfg, float *rec, int32_t *bbox, int32_t *tile_count, int32_t *isect_count,
                     void *stream);

/* ---- Rasterizer: replicate, assign tile ID, cull --------------------------
 * xpr_depth_order: order[n] = the primitives with tile_count > 0 sorted by
 * (depth, index) ascending (float bits of camera z; stable), followed by the
 * others in index order.  Emitting intersections in this order lets xpr_sort
 * sort by tile alone (begin_bit = 32) and still produce the (tile, depth)
 * order of Sec. 4.2.  workspace: >= xpr_depth_order_workspace(n) bytes,
 * 256-byte aligned. */
size_t xpr_depth_order_workspace(int64_t n);
int xpr_depth_order(const float *rec, const int32_t *tile_count, int64_t n, int32_t *order, void *workspace,
                    size_t ws_bytes, void *stream);

/* xpr_tile_bin (Sec. 4.2 Replicate / Assign tile ID / Cull): for the
 * primitive i = order[j] at each position j (order NULL = identity) and slot
 * r = 0 .. w_i h_i - 1 of its bounding box, x = xmin + r mod w_i,
 * y = ymin + r div w_i, t = y W' + x; the pair is kept iff the StopThePop cull
 * of Listing 1 tile_cull passes (decision taken in FP32 with a fixed sequence
 * of correctly rounded operations).  Culled pairs are not emitted (the
 * paper's "tile ID T" slots are dropped instead of being sorted to the end).
 * isect_count (may be NULL) is xpr_project's per-primitive count of kept
 * tiles; when NULL the counts are computed here in a separate pass.
 * Outputs: offsets[n+1] int32 (exclusive prefix sum over positions j of the
 * surviving counts; offsets[n] = total); per pair, in (position, r) order:
 * keys[total] = (t << 32) | float_bits(depth) (u64, may be NULL),
 * tiles[total] = t (u32, may be NULL; at least one of keys / tiles is
 * required) and vals[total] = primitive index; *n_isect (HOST) = total.
 * If total > capacity, returns XPR_ERR_CAPACITY with *n_isect set and the
 * pair arrays untouched (the caller re-sizes and calls again).
 * Synchronises `stream` to read the total.  workspace:
 * >= xpr_tile_bin_workspace(n) bytes, 256-byte aligned. */
size_t xpr_tile_bin_workspace(int64_t n);
int xpr_tile_bin(const float *rec, const int32_t *bbox, const int32_t *tile_count, const int32_t *isect_count,
                 const int32_t *order, int64_t n, const XprCamera *cam, const XprConfig *cfg, int32_t *offsets,
                 uint64_t *keys, uint32_t *tiles, uint32_t *vals, int64_t capacity, int64_t *n_isect,
                 void *workspace, size_t ws_bytes, void *stream);

/* xpr_tile_bin_noalloc: xpr_tile_bin without a workspace argument, for callers
 * that cannot allocate device memory (for example a process whose device
 * memory belongs to another framework's pool, or a latency-critical loop that
 * must not call cudaMalloc/cudaFree because they can synchronise the device).
 * The paper has no counterpart; this is a convenience of the library.
 * Scratch: a file-scope __device__ array of 131,328 bytes inside libxpr.so,
 * held by every GPU that loads the library until the process exits.
 * Limit: n <= 67,108,864 primitives; larger n returns XPR_ERR_INVALID.
 * The first call on each device looks up the array's device address
 * (cudaGetSymbolAddress, with that device current) and caches it; make that
 * first call before any stream capture.  Every call shares the array: nothing
 * in it needs to start at zero (each call writes all it reads), but calls that
 * overlap on the GPU (different streams, or different host threads on one
 * device) race on it and must be serialised by the caller.  Allocates nothing;
 * arguments, outputs and errors are those of xpr_tile_bin. */
int xpr_tile_bin_noalloc(const float *rec, const int32_t *bbox, const int32_t *tile_count,
                         const int32_t *isect_count, const int32_t *order, int64_t n, const XprCamera *cam,
                         const XprConfig *cfg, int32_t *offsets, uint64_t *keys, uint32_t *tiles, uint32_t *vals,
                         int64_t capacity, int64_t *n_isect, void *stream);

/* ---- Rasterizer: sort and identify bounds ---------------------------------
 * xpr_sort (Sec. 4.2 "Sort and identify bounds"): stable LSD radix sort of
 * (key, val) by key bits [begin_bit, 32 + ceil(log2(n_tiles))), then
 * ranges[t] = [start, end) of tile t's segment ([0,0) for empty tiles).
 * begin_bit = 0 sorts the full (tile, depth) key; begin_bit = 32 sorts by tile
 * only and equals the full sort when the input is already in depth order
 * (xpr_tile_bin with the xpr_depth_order permutation): 2 passes instead of 6
 * at 8160 tiles.  Stability keeps equal keys in input order.
 * keys_in/vals_in are read only and must not alias keys_out/vals_out.
 * workspace: >= xpr_sort_workspace(n_isect, n_tiles) bytes, 256-byte aligned. */
size_t xpr_sort_workspace(int64_t n_isect, int32_t n_tiles);
int xpr_sort(const uint64_t *keys_in, const uint32_t *vals_in, int64_t n_isect, int32_t n_tiles, int32_t begin_bit,
             uint64_t *keys_out, uint32_t *vals_out, int32_t *ranges, void *workspace, size_t ws_bytes,
             void *stream);

/* xpr_sort_tiles: the same stable sort and segment bounds for pairs given as
 * u32 tile ids (xpr_tile_bin's `tiles` output) instead of u64 keys; with pairs
 * emitted in xpr_depth_order order the result is the (tile, depth) order of
 * Sec. 4.2 while moving 8 instead of 12 bytes per pair and pass.
 * tiles_out may be NULL when only vals_out and ranges are wanted: the last
 * pass then writes no tile ids, and with more than two 8-bit passes
 * (n_tiles > 65536) tiles_in is overwritten (used as the second key buffer).
 * tiles_in/vals_in must not alias tiles_out/vals_out.  workspace:
 * >= xpr_sort_tiles_workspace(n_isect, n_tiles) bytes, 256-byte aligned. */
size_t xpr_sort_tiles_workspace(int64_t n_isect, int32_t n_tiles);
int xpr_sort_tiles(const uint32_t *tiles_in, const uint32_t *vals_in, int64_t n_isect, int32_t n_tiles,
                   uint32_t *tiles_out, uint32_t *vals_out, int32_t *ranges, void *workspace, size_t ws_bytes,
                   void *stream);

/* ---- Shader ----------------------------------------------------------------
 * xpr_render_fwd (Sec. 2 Shader, Algorithm 1, Listing 1 evaluate): one thread
 * block per tile walks vals[ranges[t,0]:ranges[t,1]] front to back for each
 * pixel (x, y): d = (x, y) - mu_2D, power = -(c00 dx^2 + 2 c01 dx dy +
 * c11 dy^2)/2; skip if power > 0; alpha = min(alpha_max, o exp(power)); skip
 * if alpha < alpha_thresh; stop if T (1 - alpha) < t_eps; else C += rgb alpha T,
 * T *= 1 - alpha.  Finally C += T bg.
 * Outputs: image[3,H,W] (planar), t_final[H,W], n_contrib[H,W] int32 (1 +
 * position in the tile's list of the last blended entry; 0 if none). */
int xpr_render_fwd(const float *rec, int64_t n, const uint32_t *vals, const int32_t *ranges, const XprCamera *cam,
                   const XprConfig *cfg, float *image, float *t_final, int32_t *n_contrib, void *stream);

/* ---- Adjoint ---------------------------------------------------------------
 * xpr_render_bwd: adjoint of xpr_render_fwd given d_image[3,H,W] = dL/dimage
 * and the forward's t_final / n_contrib.  Each tile is re-walked back to front
 * from n_contrib, recomputing T_i = T_{i+1} / (1 - alpha_i) instead of storing
 * per-pixel lists; dL/drgb_i = alpha_i T_i g, dL/dalpha_i = g.(rgb_i T_i -
 * S_i / (1 - alpha_i)) with S_i the colour behind i (including T_final bg),
 * zero through the alpha_max clamp.  Per-primitive gradients are reduced over
 * each warp and thread block before one set of atomics per (tile, primitive).
 * d_rec[n,12] is OVERWRITTEN with the screen-space gradients (layout above).
 * If prims and d_prims are both non-NULL, the projection adjoint is applied
 * too and d_prims (all five arrays) is OVERWRITTEN with dL/d(mu, scale, quat,
 * opacity, sh); invisible primitives get zeros. */
int xpr_render_bwd(const float *rec, int64_t n, const uint32_t *vals, const int32_t *ranges, const XprCamera *cam,
                   const XprConfig *cfg, const float *t_final, const int32_t *n_contrib, const float *d_image,
                   float *d_rec, const XprPrims *prims, const XprPrimsGrad *d_prims, void *stream);

/* xpr_project_bwd: the projection adjoint alone (screen-space d_rec -> d_prims,
 * all five arrays overwritten).  Same math as the second half of
 * xpr_render_bwd. */
int xpr_project_bwd(const XprPrims *prims, int64_t n, const XprCamera *cam, const XprConfig *cfg,
                    const float *d_rec, const XprPrimsGrad *d_prims, void *stream);

/* ---- Multi-view (batched) form ----------------------------------------------
 * V = n_views (1..16) views of one scene of n primitives in one launch per
 * stage.  Records are view-major: record v * n + i is primitive i seen from
 * view v (rec[V*n,12], bbox[V*n,4], tile_count[V*n], isect_count[V*n]).
 * All views of a render call share cam->width/height and the tile size; tile
 * t of view v has global id v * T + t (T tiles per view), images are
 * [V,3,H,W], t_final and n_contrib [V,H,W].  Every stage computes exactly what
 * the single-view call computes for each view; only the scheduling differs:
 *   xpr_project_views reads each primitive's parameters once for all views
 *     (cams: HOST array of V cameras);
 *   xpr_depth_order_views orders records by (view, depth, index);
 *   xpr_tile_bin_views emits u32 global tile ids (tiles) and record indices
 *     (vals) in that order;
 *   xpr_sort_tiles with n_tiles = V * T gives the per-tile segments;
 *   xpr_tile_worklist lists tiles by descending segment length, and the
 *     render calls, given that list and a device int32 counter, run one
 *     persistent grid whose blocks take tiles from it through the counter
 *     (the paper's trip-count binning of Sec. 4.3 made dynamic); with
 *     worklist NULL they launch one block per tile;
 *   xpr_project_bwd_views sums the adjoint over views into d_prims. */
int xpr_project_views(const XprPrims *prims, int64_t n, const XprCamera *cams, int32_t n_views, const XprConfig *cfg,
                      float *rec, int32_t *bbox, int32_t *tile_count, int32_t *isect_count, void *stream);
int xpr_depth_order_views(const float *rec, const int32_t *tile_count, int64_t n, int32_t n_views, int32_t *order,
                          void *workspace, size_t ws_bytes, void *stream); /* workspace: xpr_depth_order_workspace(V*n) */
int xpr_tile_bin_views(const float *rec, const int32_t *bbox, const int32_t *tile_count, const int32_t *isect_count,
                       const int32_t *order, int64_t n, int32_t n_views, const XprCamera *cam, const XprConfig *cfg,
                       int32_t *offsets, uint32_t *tiles, uint32_t *vals, int64_t capacity, int64_t *n_isect,
                       void *workspace, size_t ws_bytes, void *stream); /* offsets[V*n+1]; workspace: xpr_tile_bin_workspace(V*n) */
size_t xpr_tile_worklist_workspace(int32_t n_tiles);
int xpr_tile_worklist(const int32_t *ranges, int32_t n_tiles, int32_t *worklist, void *workspace, size_t ws_bytes,
                      void *stream);
int xpr_render_fwd_views(const float *rec, int64_t n, int32_t n_views, const uint32_t *vals, const int32_t *ranges,
                         const XprCamera *cam, const XprConfig *cfg, float *image, float *t_final, int32_t *n_contrib,
                         const int32_t *worklist, int32_t *counter, void *stream);
int xpr_render_bwd_views(const float *rec, int64_t n, int32_t n_views, const uint32_t *vals, const int32_t *ranges,
                         const XprCamera *cam, const XprConfig *cfg, const float *t_final, const int32_t *n_contrib,
                         const float *d_image, float *d_rec, const int32_t *worklist, int32_t *counter,
                         void *stream); /* d_rec[V*n,12] overwritten */
int xpr_project_bwd_views(const XprPrims *prims, int64_t n, const XprCamera *cams, int32_t n_views,
                          const XprConfig *cfg, const float *d_rec, const XprPrimsGrad *d_prims, void *stream);

/* ---- Multi-scene batched form (3DGS) -------------------------------------------
 * K items (1 <= K <= 16), each a (scene, camera) pair with its own primitive
 * count and image size (XprItem), run through one launch per stage; per item
 * the result is exactly what the single-view calls compute for that scene and
 * camera (records, sorted lists, image, gradients), so a batch can mix scenes
 * of uneven size and requests of different resolutions (the paper's
 * trip-count binning, Sec. 4.3, made dynamic over all items' tiles).
 * cams, items: HOST arrays of K entries; R = the records of all items
 * (the last rec_offset + its padded size).
 *   xpr_project_items: rec[R,12], bbox[R,4], tile_count[R] (padding records
 *     invisible, tile count 0);
 *   xpr_depth_order_items: order[R]: each item's records by (depth key,
 *     index), those without tiles last, item k's at [rec_offset, + padded n);
 *     workspace: xpr_depth_order_workspace(R);
 *   xpr_bin_sorted_items: as xpr_bin_sorted over all items: ranges[S,2] for
 *     S = the last tile_offset + its tiles, vals[capacity], *n_isect (HOST);
 *     synchronises the stream once; workspace: xpr_bin_sorted_items_workspace;
 *   xpr_render_fwd_items / xpr_render_bwd_items: as the _views calls with a
 *     work list over all S tiles (xpr_tile_worklist) or NULL (one block per
 *     tile); d_rec[R,12] overwritten;
 *   xpr_project_bwd_items: d_prims (concatenated layout) OVERWRITTEN with the
 *     sum over items of each scene primitive's gradient. */
int xpr_project_items(const XprPrims *prims, const XprCamera *cams, const XprItem *items, int32_t n_items,
                      const XprConfig *cfg, float *rec, int32_t *bbox, int32_t *tile_count, void *stream);
int xpr_depth_order_items(const float *rec, const int32_t *tile_count, const XprItem *items, int32_t n_items,
                          int32_t *order, void *workspace, size_t ws_bytes, void *stream);
size_t xpr_bin_sorted_items_workspace(const XprCamera *cams, const XprItem *items, int32_t n_items,
                                      const XprConfig *cfg);
int xpr_bin_sorted_items(const float *rec, const int32_t *bbox, const int32_t *tile_count, const int32_t *order,
                         const XprCamera *cams, const XprItem *items, int32_t n_items, const XprConfig *cfg,
                         int32_t *ranges, uint32_t *vals, int64_t capacity, int64_t *n_isect, void *workspace,
                         size_t ws_bytes, void *stream);
int xpr_render_fwd_items(const float *rec, const uint32_t *vals, const int32_t *ranges, const XprCamera *cams,
                         const XprItem *items, int32_t n_items, const XprConfig *cfg, float *image, float *t_final,
                         int32_t *n_contrib, const int32_t *worklist, int32_t *counter, void *stream);
int xpr_render_bwd_items(const float *rec, const uint32_t *vals, const int32_t *ranges, const XprCamera *cams,
                         const XprItem *items, int32_t n_items, const XprConfig *cfg, const float *t_final,
                         const int32_t *n_contrib, const float *d_image, float *d_rec, const int32_t *worklist,
                         int32_t *counter, void *stream);
int xpr_project_bwd_items(const XprPrims *prims, int64_t n_prims, const XprCamera *cams, const XprItem *items,
                          int32_t n_items, const XprConfig *cfg, const float *d_rec, const XprPrimsGrad *d_prims,
                          void *stream);

/* xpr_forward_items: the whole forward of a multi-scene batch in one call (the
 * serving runtime's entry point): the items' projection with the exact
 * kept-tile counts, xpr_depth_order_items, the binning and tile sort by rows
 * of xpr_bin_rows_items when every item's grid has at most 128 x 128 tiles
 * (else, or when the span slots outgrow the workspace's room for
 * capacity / 2 + R of them, the offsets scan, the emission of (global tile
 * id, record) pairs in depth order as xpr_tile_bin, and xpr_sort_tiles over
 * all items' tiles: the same lists either way), xpr_tile_worklist and
 * xpr_render_fwd_items with the work list (one block per tile for a single
 * item; the same lists and images as the staged calls), every intermediate
 * carved from one
 * caller-owned workspace
 * (device, 256-byte aligned) of xpr_forward_items_workspace(cams, items, K,
 * cfg, capacity) bytes, where capacity is the room for intersection pairs.
 * Outputs as xpr_render_fwd_items: image[3 * pixels], t_final[pixels],
 * n_contrib[pixels] (device).  *n_isect (HOST) receives the pair count; if it
 * exceeds capacity the call returns XPR_ERR_CAPACITY before rendering (call
 * again with a workspace sized for at least that many pairs).  Synchronises
 * the stream once (the pair count). */
size_t xpr_forward_items_workspace(const XprCamera *cams, const XprItem *items, int32_t n_items, const XprConfig *cfg,
                                   int64_t capacity);
int xpr_forward_items(const XprPrims *prims, const XprCamera *cams, const XprItem *items, int32_t n_items,
                      const XprConfig *cfg, float *image, float *t_final, int32_t *n_contrib, int64_t capacity,
                      int64_t *n_isect, void *workspace, size_t ws_bytes, void *stream);

/* xpr_project_color: the view-dependent colour of Listing 1 project (the SH
 * part of compute_color) for records already projected with prims->sh NULL:
 * for every visible record v * n + i (rec[.,11] != 0), rec[.,6..8] =
 * max(0, 0.5 + sum_k sh[i,k,:] Y_k(d)), d = unit vector from camera v's centre
 * to mu[i]; invisible records are not touched.  mu[n,3], sh[n,K,3] (device);
 * cams: HOST array of n_views cameras (1..16); rec[n_views*n,12] (device). */
int xpr_project_color(const float *mu, const float *sh, int64_t n, const XprCamera *cams, int32_t n_views,
                      const XprConfig *cfg, float *rec, void *stream);

/* ---- Fused bin + sort ---------------------------------------------------------
 * xpr_bin_sorted: Sec. 4.2's replicate / assign tile id / cull followed by
 * "sort and identify bounds", with no key array: it writes the sorted record
 * indices and the tile segments directly.  The result is bit-identical to
 * xpr_tile_bin (in the same emission order) followed by xpr_sort_tiles: the
 * same kept pairs (same FP32 cull), each tile's list in emission order.
 *   rec, bbox, tile_count: from xpr_project (_views), n records per view;
 *   order[V*n]: the emission order, from xpr_depth_order (_views) (record
 *     indices, view-major);
 *   ranges[V*T,2] (int32, device): OVERWRITTEN, tile t of view v at v*T + t,
 *     [0, 0) for a tile with no pairs (as xpr_sort_tiles);
 *   vals[capacity] (u32, device): record indices, tile-major, in emission order
 *     within a tile;
 *   *n_isect (HOST): the number of kept pairs I.  If I > capacity the call
 *     returns XPR_ERR_CAPACITY without writing vals (ranges are already valid
 *     for I pairs); call again with capacity >= I.
 * The call synchronises the stream once (to read I).  It does a counting pass,
 * a prefix over a (chunk x tile) count matrix and a writing pass; every tile's
 * segment is [start, end) of vals.  The passes walk the emission positions in
 * chunks, 8 tile rows per thread block, each row's kept span of tile columns
 * from the row form of the cull; grids with more than 4096 tile columns are
 * rejected with XPR_ERR_INVALID (use xpr_tile_bin + xpr_sort_tiles for them).
 * workspace (device, 256-byte aligned, caller-owned):
 * xpr_bin_sorted_workspace(n, V, cam, cfg) bytes (the count matrix holds at
 * most 16M entries), 0 for invalid arguments. */
size_t xpr_bin_sorted_workspace(int64_t n, int32_t n_views, const XprCamera *cam, const XprConfig *cfg);
int xpr_bin_sorted(const float *rec, const int32_t *bbox, const int32_t *tile_count, const int32_t *order, int64_t n,
                   int32_t n_views, const XprCamera *cam, const XprConfig *cfg, int32_t *ranges, uint32_t *vals,
                   int64_t capacity, int64_t *n_isect, void *workspace, size_t ws_bytes, void *stream);

/* ---- Bin + sort by tile rows ------------------------------------------------
 * xpr_bin_rows: Sec. 4.2's replicate / assign tile id / cull and "sort and
 * identify bounds" for one view whose tile grid has at most 128 columns and
 * 128 rows, with no radix pass over the pairs: the row form of the cull gives
 * every primitive one span of kept tile columns per row of its box; the spans
 * (about seven pairs each on the headline workload) are written grouped by row
 * in depth order (their places from a scanned count of box rows per row and
 * chunk of depth positions), and a stable pass by tile column places every
 * span's pairs straight into the tile-major lists (a column histogram per
 * window of 3968 pairs, its scan, ranks from the spans covering each column).
 * Every tile's list is bit-identical to
 * xpr_tile_bin in the same order followed by xpr_sort_tiles: the same kept
 * pairs (same FP32 cull), each tile's list in emission order; the tiles'
 * segments lie in column-major tile order (the ranges locate them).
 *   rec, bbox, tile_count: from xpr_project (n records of one view);
 *   isect_count[n] (device, may be NULL): the kept tile counts from
 *     xpr_project; with them the call reads both totals back at once;
 *   order[n]: the emission order, from xpr_depth_order;
 *   ranges[T,2] (int32, device): OVERWRITTEN, [0, 0) for a tile with no pairs;
 *   vals[capacity] (u32, device): record indices, each tile's list contiguous
 *     and in emission order;
 *   *n_isect, *n_spans (HOST): the kept pairs I and the span slots S (one per
 *     row of every box).  If I > capacity or workspace_bytes is below
 *     xpr_bin_rows_workspace(n, S, I, cam, cfg), the call returns
 *     XPR_ERR_CAPACITY with both counts set and without writing vals or
 *     ranges; call again with enough of both.
 * The counts are read back at two points (the span total, and the pair
 * total: with the span total when isect_count is given, else from the
 * emission).  When the workspace holds room for `capacity` pairs and some
 * span slots, the host waits for each count through an event while the
 * kernels that do not need it are already queued (the emission is bounded by
 * that room); otherwise it synchronises the stream before the work that
 * needs the count.  Grids with more than 128 tile columns or rows are rejected with
 * XPR_ERR_INVALID (use xpr_tile_bin + xpr_sort_tiles for them).
 * workspace (device, 256-byte aligned, caller-owned):
 * xpr_bin_rows_workspace(n, S, I, cam, cfg) bytes (0 for invalid arguments);
 * with S = I = 0 it is the least size that lets the call report the counts. */
size_t xpr_bin_rows_workspace(int64_t n, int64_t n_spans, int64_t n_isect, const XprCamera *cam,
                              const XprConfig *cfg);
int xpr_bin_rows(const float *rec, const int32_t *bbox, const int32_t *tile_count, const int32_t *isect_count,
                 const int32_t *order, int64_t n, const XprCamera *cam, const XprConfig *cfg, int32_t *ranges,
                 uint32_t *vals, int64_t capacity, int64_t *n_isect, int64_t *n_spans, void *workspace,
                 size_t workspace_bytes, void *stream);

/* xpr_bin_rows_views / xpr_bin_rows_items: xpr_bin_rows over a batch (the
 * multi-view and multi-scene forms, Sec. 4.3), every grid at most 128 x 128
 * tiles: each view's or item's lists are bit-identical to xpr_tile_bin_views
 * (or the items' emission) followed by xpr_sort_tiles over all S tiles.  The
 * spans carry their item, the pass by column groups the pairs by (column, row,
 * item), and the tiles' segments lie in that order (the ranges locate them).
 *   _views: V = n_views (1..16) views of n primitives, records view-major
 *     (rec[V*n,12] ... from xpr_project_views, isect_count[V*n] or NULL,
 *     order[V*n] from xpr_depth_order_views); ranges[V*T,2];
 *   _items: K items (1..16; cams and items HOST arrays as in
 *     xpr_project_items), R records from xpr_project_items (isect_count[R] or
 *     NULL), order[R] from xpr_depth_order_items; ranges[S,2], S = the last
 *     tile_offset + its tiles.
 * Counts, capacity protocol, synchronisation and errors as xpr_bin_rows (the
 * workspace functions take the same batch description; 0 for invalid
 * arguments). */
size_t xpr_bin_rows_views_workspace(int64_t n, int32_t n_views, int64_t n_spans, int64_t n_isect,
                                    const XprCamera *cam, const XprConfig *cfg);
int xpr_bin_rows_views(const float *rec, const int32_t *bbox, const int32_t *tile_count, const int32_t *isect_count,
                       const int32_t *order, int64_t n, int32_t n_views, const XprCamera *cam, const XprConfig *cfg,
                       int32_t *ranges, uint32_t *vals, int64_t capacity, int64_t *n_isect, int64_t *n_spans,
                       void *workspace, size_t workspace_bytes, void *stream);
size_t xpr_bin_rows_items_workspace(const XprCamera *cams, const XprItem *items, int32_t n_items,
                                    const XprConfig *cfg, int64_t n_spans, int64_t n_isect);
int xpr_bin_rows_items(const float *rec, const int32_t *bbox, const int32_t *tile_count, const int32_t *isect_count,
                       const int32_t *order, const XprCamera *cams, const XprItem *items, int32_t n_items,
                       const XprConfig *cfg, int32_t *ranges, uint32_t *vals, int64_t capacity, int64_t *n_isect,
                       int64_t *n_spans, void *workspace, size_t workspace_bytes, void *stream);

/* ---- Rendered features (3DGS) ----------------------------------------------------
 * The "rendered feature" class of the design space (depth, semantics): channel c of
 * pixel p is sum_i f_ic alpha_i T_i over the same contributors and weights as the
 * colour, with zero background.  feat[n, n_feat] (device, row-major; may be NULL when
 * n_feat == 0) holds the per-primitive feature rows; with_depth != 0 appends one
 * channel whose per-primitive value is the record's depth (camera z), i.e. the
 * expected depth.  1 <= n_feat + with_depth <= 16.
 * xpr_render_fwd_feat: as xpr_render_fwd (same image bit for bit) plus
 *   features[n_feat + with_depth, H, W].
 * xpr_render_bwd_feat: the adjoint for d_image[3,H,W] and d_features[n_feat +
 *   with_depth, H, W]: d_rec[n,12] (OVERWRITTEN; record layout, the depth
 *   channel's gradient in entry 9, which xpr_project_bwd takes through camera z)
 *   and d_feat[n, n_feat] (OVERWRITTEN; may be NULL when n_feat == 0). */
int xpr_render_fwd_feat(const float *rec, int64_t n, const float *feat, int32_t n_feat, int32_t with_depth,
                        const uint32_t *vals, const int32_t *ranges, const XprCamera *cam, const XprConfig *cfg,
                        float *image, float *features, float *t_final, int32_t *n_contrib, void *stream);
int xpr_render_bwd_feat(const float *rec, int64_t n, const float *feat, int32_t n_feat, int32_t with_depth,
                        const uint32_t *vals, const int32_t *ranges, const XprCamera *cam, const XprConfig *cfg,
                        const float *t_final, const int32_t *n_contrib, const float *d_image,
                        const float *d_features, float *d_rec, float *d_feat, void *stream);

/* ---- 3DGUT (cfg->method == XPR_METHOD_3DGUT) ------------------------------------
 * The 3DGUT instance of project / tile_cull / pixel_info / evaluate (Sec. 3
 * method examples; Appendix, implementation of XPR-3DGUT).  Depth order,
 * binning and sorting are the 3DGS entry points, called with the same config:
 * its method field switches the tile cull to the ray-offset bounds (tile max
 * bounds + 1, pixel centres at +0.5).  The projection / render entry points
 * above refuse a 3DGUT config and these refuse a 3DGS one (XPR_ERR_INVALID).
 *
 * Shader data, 16 floats per record (this library's form of the paper's
 * p_sd = (o_c, M, o', c), chosen so that float32 evaluation does not cancel):
 *   [0] p0.x [1] p0.y  projected centre (fx x/z + cx, fy y/z + cy)
 *   [2..4] A_0 = (z/fx) M W^T e_0   [5..7] A_1 = (z/fy) M W^T e_1
 *   [8..10] o_c = M (c - mu)   [11] o' (Mip-Splatting opacity)
 *   [12..14] rgb   [15] |o_c|^2
 * with M = S^-1 R^T, W the world-to-camera rotation, c the camera centre.
 * Pixel (x, y) is evaluated on the ray through (x + 0.5, y + 0.5); with
 * (dx, dy) = (x + 0.5, y + 0.5) - p0, a = dx A_0 + dy A_1, b = a - o_c, the
 * largest response along the ray is G = exp(-(|a|^2 - (a.b)^2 / |b|^2) / 2),
 * equal to the paper's exp(-|o_c + tau_max d_c|^2 / 2).  Gradients d_sd use
 * the same layout (entry 15 stays 0: |o_c|^2 is folded into d o_c). */
#define XPR_SD_FLOATS 16

/* xpr_project_ut: unscented-transform projection of n primitives.  Seven
 * sigma points mu, mu +- sqrt(3) s_a R e_a (UT alpha = 1, beta = 2, kappa = 0:
 * mean weights 0 and 1/6, covariance weights 2 and 1/6) through the pinhole
 * projection give mu_2D and Sigma_2D; dilation + cov_dilation I; o' = o
 * sqrt(det_0 / det); conic, extents sqrt(2 ln(o'/a_t) Sigma_2D,xx) (and yy),
 * tile box of mu_2D - 0.5.  Invisible when a sigma point has camera z <=
 * z_near, det <= 0, o' <= alpha_thresh, r = 0 or tc = 0.  Outputs rec[n,12]
 * (3DGS layout: UT mean and conic, o', rgb, depth, ln(o'/a_t), visible),
 * sd[n,16], bbox[n,4], tile_count[n], isect_count[n] (may be NULL) as
 * xpr_project.  prims->sh must not be NULL.  rec, sd, bbox, quat 16-byte
 * aligned. */
int xpr_project_ut(const XprPrims *prims, int64_t n, const XprCamera *cam, const XprConfig *cfg, float *rec,
                   float *sd, int32_t *bbox, int32_t *tile_count, int32_t *isect_count, void *stream);

/* xpr_render_ut_fwd: front-to-back compositing of the sorted lists (as
 * xpr_render_fwd) with the 3DGUT evaluate: alpha = min(alpha_max, o' G),
 * valid iff G > 0.0113, skipped if alpha < alpha_thresh.  sd[n,16] from
 * xpr_project_ut; vals, ranges from xpr_sort_tiles / xpr_bin_sorted;
 * outputs image[3,H,W], t_final[H,W], n_contrib[H,W].  Tiles of 8 or 16. */
int xpr_render_ut_fwd(const float *sd, int64_t n, const uint32_t *vals, const int32_t *ranges, const XprCamera *cam,
                      const XprConfig *cfg, float *image, float *t_final, int32_t *n_contrib, void *stream);

/* xpr_render_ut_bwd: reverse-order adjoint of xpr_render_ut_fwd.  d_sd[n,16]
 * is OVERWRITTEN (zeroed, then accumulated with atomics). */
int xpr_render_ut_bwd(const float *sd, int64_t n, const uint32_t *vals, const int32_t *ranges, const XprCamera *cam,
                      const XprConfig *cfg, const float *t_final, const int32_t *n_contrib, const float *d_image,
                      float *d_sd, void *stream);

/* xpr_project_ut_bwd: adjoint of xpr_project_ut from d_sd[n,16] to the
 * parameter gradients (OVERWRITTEN; zero for invisible primitives), the
 * Mip-Splatting factor differentiated through the unscented covariance. */
int xpr_project_ut_bwd(const XprPrims *prims, int64_t n, const XprCamera *cam, const XprConfig *cfg,
                       const float *d_sd, const XprPrimsGrad *d_prims, void *stream);

/* 3DGUT, multi-view form (as the 3DGS _views entry points): V <= 16 cameras of
 * one image size; records and shader data are view-major [V*n, ...]; tile t
 * of view v is v*T + t in the binning, the sort and ranges[V*T,2]; images
 * [V,3,H,W].  worklist (may be NULL) / counter: a persistent render grid
 * taking tiles from xpr_tile_worklist's order through *counter (zeroed by the
 * call).  d_sd[V*n,16] is OVERWRITTEN; the projection adjoint sums the views'
 * gradients. */
int xpr_project_ut_views(const XprPrims *prims, int64_t n, const XprCamera *cams, int32_t n_views,
                         const XprConfig *cfg, float *rec, float *sd, int32_t *bbox, int32_t *tile_count,
                         int32_t *isect_count, void *stream);
int xpr_render_ut_fwd_views(const float *sd, int64_t n, int32_t n_views, const uint32_t *vals, const int32_t *ranges,
                            const XprCamera *cam, const XprConfig *cfg, float *image, float *t_final,
                            int32_t *n_contrib, const int32_t *worklist, int32_t *counter, void *stream);
int xpr_render_ut_bwd_views(const float *sd, int64_t n, int32_t n_views, const uint32_t *vals, const int32_t *ranges,
                            const XprCamera *cam, const XprConfig *cfg, const float *t_final,
                            const int32_t *n_contrib, const float *d_image, float *d_sd, const int32_t *worklist,
                            int32_t *counter, void *stream);
int xpr_project_ut_bwd_views(const XprPrims *prims, int64_t n, const XprCamera *cams, int32_t n_views,
                             const XprConfig *cfg, const float *d_sd, const XprPrimsGrad *d_prims, void *stream);

/* ---- LinPrim (cfg->method == XPR_METHOD_LINPRIM) -------------------------------
 * Octahedra {x : ||S^-1 R^T (x - mu)||_1 <= 1} with homogeneous density (Appendix,
 * implementation of XPR-LinPrim).  Parameters as XprPrims with scale the three
 * half-extents and opacity o; sigma = -log(1 - 0.99 clip(o, 0, 0.999)) / (2 min s).
 * Projection: A = J3 W R diag(s) (J3 = pinhole Jacobian plus the row m_c / |m_c|
 * of the Euclidean distance), c0, c1, c2 = rows of A^-1, slab normals
 * n_i = c0 + e1 c1 + e2 c2 for (e1, e2) in (+,+), (+,-), (-,+), (-,-).
 * Shader data, 20 floats per record (also the cull's data):
 *   [0] mu_2D.x [1] mu_2D.y [2] sigma [3] -log(1 - alpha_thresh)
 *   [4 + 3i .. 6 + 3i] slab i: (n_x / n_z, n_y / n_z, 1 / |n_z|) (0, 0, +inf when |n_z| < 1e-10)
 *   [16..18] rgb [19] 0
 * Record (rec[12]): mu_2D [0,1], rgb [6..8], Euclidean depth |m_c| [9], visible [11], rest 0;
 * xpr_depth_order reads it as for 3DGS.  Pixel (x, y) is evaluated at (x + 0.5, y + 0.5):
 * with (dX, dY) its offset from mu_2D, slab i admits tau in m_i -+ h_i,
 * m_i = -(p_i dX + q_i dY); dtau = min (m + h) - max (m - h); alpha = 1 - exp(-sigma dtau)
 * when dtau > 0 (then the framework's clamp, gate and T_eps as for 3DGS).
 * Gradients d_sd use the shader-data layout ([3] and [19] stay 0). */
#define XPR_LP_SD_FLOATS 20

/* xpr_project_lp: extents ex = max_k |A_0k|, ey = max_k |A_1k| (the six
 * vertices), tile box of mu_2D - 0.5 as 3DGUT; visible iff camera z > z_near,
 * |m_c| > z_near, min s > 0, r > 0, tc > 0.  Outputs rec[n,12], sd[n,20],
 * bbox[n,4], tile_count[n], isect_count[n] (may be NULL: kept tiles of the
 * box under xpr_tile_bin_lp's cull).  prims->sh must not be NULL; rec, sd,
 * bbox, quat 16-byte aligned. */
int xpr_project_lp(const XprPrims *prims, int64_t n, const XprCamera *cam, const XprConfig *cfg, float *rec,
                   float *sd, int32_t *bbox, int32_t *tile_count, int32_t *isect_count, void *stream);

/* xpr_tile_bin_lp: xpr_tile_bin for LinPrim.  The cull keeps a (primitive,
 * tile) pair iff sigma dtau_upper >= -log(1 - alpha_thresh), dtau_upper the
 * per-tile chord bound of Eq. (linprim_tile_cull) over the tile's four
 * pixel-centre corners (inclusive pixel bounds + 0.5), decided in FP32 from
 * sd with one correctly rounded operation per step.  Arguments, capacity
 * protocol and outputs as xpr_tile_bin, plus sd[n,20] from xpr_project_lp. */
int xpr_tile_bin_lp(const float *rec, const float *sd, const int32_t *bbox, const int32_t *tile_count,
                    const int32_t *isect_count, const int32_t *order, int64_t n, const XprCamera *cam,
                    const XprConfig *cfg, int32_t *offsets, uint64_t *keys, uint32_t *tiles, uint32_t *vals,
                    int64_t capacity, int64_t *n_isect, void *workspace, size_t ws_bytes, void *stream);

/* xpr_render_lp_fwd / xpr_render_lp_bwd: compositing of the sorted lists with
 * the LinPrim evaluate, and its reverse-order adjoint (d_sd[n,20] OVERWRITTEN). */
int xpr_render_lp_fwd(const float *sd, int64_t n, const uint32_t *vals, const int32_t *ranges, const XprCamera *cam,
                      const XprConfig *cfg, float *image, float *t_final, int32_t *n_contrib, void *stream);
int xpr_render_lp_bwd(const float *sd, int64_t n, const uint32_t *vals, const int32_t *ranges, const XprCamera *cam,
                      const XprConfig *cfg, const float *t_final, const int32_t *n_contrib, const float *d_image,
                      float *d_sd, void *stream);

/* xpr_project_lp_bwd: adjoint of xpr_project_lp from d_sd[n,20] to the
 * parameter gradients (OVERWRITTEN; zero for invisible primitives). */
int xpr_project_lp_bwd(const XprPrims *prims, int64_t n, const XprCamera *cam, const XprConfig *cfg,
                       const float *d_sd, const XprPrimsGrad *d_prims, void *stream);

/* ---- Misc ------------------------------------------------------------------ */
const char *xpr_status_string(int status);
const char *xpr_last_error(void); /* message of the last failing call on this host thread */
int xpr_version(void);
/* Number of kernels this library has launched in the process so far (all threads). */
unsigned long long xpr_launch_count(void);
/* xpr_device_check: synchronises the current device, then reads and clears the
 * error flags that the library's kernels record there instead of faulting.
 * The sort's chained scan (xpr_sort, xpr_sort_tiles, xpr_depth_order and the
 * entries built on them) waits on words that earlier blocks publish; each wait
 * is bounded, and a wait that gives up sets the timeout flag.  A published word
 * that cannot be right, or an output position outside the buffer (the write is
 * skipped), sets the consistency flag.  Returns XPR_OK when neither flag was
 * set since the last call, else XPR_ERR_TIMEOUT or XPR_ERR_INTERNAL (the
 * results of the calls in between are then unreliable). */
int xpr_device_check(void);
/* xpr_selftest_wait: exercises the bounded wait of the sort's chained scan
 * against words that nothing publishes.  `zeroed` is a device buffer of at
 * least 512 uint32 whose first 256 are zero; one block of 256 threads looks
 * back at them, gives up after `polls` polls each (1..2^20) and records the
 * timeout, so the next xpr_device_check returns XPR_ERR_TIMEOUT.  Words
 * 256..511 receive the (short) counts.  The device stays usable. */
int xpr_selftest_wait(uint32_t *zeroed, int32_t polls, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* XPR_H */
