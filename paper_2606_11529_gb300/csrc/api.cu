// C-ABI entry points of libxpr (declared in include/xpr.h): argument validation, workspace
// carving and launches on the caller's stream.  No device memory is allocated here.
#include <stdarg.h>
#include <stdio.h>

#include <atomic>

#include <algorithm>

#include "xpr_internal.cuh"

namespace xpr {

static thread_local char g_err[512] = "";
static std::atomic<unsigned long long> g_launches{0};

void set_error(const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}

int fail(int status, const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return status;
}

int check_launch(const char *what) {
    g_launches.fetch_add(1, std::memory_order_relaxed);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(XPR_ERR_CUDA, "%s launch failed: %s", what, cudaGetErrorString(e));
    return XPR_OK;
}

static bool aligned(const void *p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

int validate_camera_config(const XprCamera *cam, const XprConfig *cfg) {
    if (!cam || !cfg) return fail(XPR_ERR_INVALID, "camera/config pointer is NULL");
    if (cam->width < 1 || cam->height < 1 || cam->width > 32768 || cam->height > 32768)
        return fail(XPR_ERR_INVALID, "image size %dx%d out of range [1, 32768]", cam->width, cam->height);
    if (cam->model != 0 && cam->model != 1)
        return fail(XPR_ERR_INVALID, "camera model %d not supported (0 = pinhole, 1 = fisheye)", cam->model);
    if (!(cam->fx > 0.f) || !(cam->fy > 0.f)) return fail(XPR_ERR_INVALID, "focal lengths must be positive");
    if ((cfg->tile_w != 8 && cfg->tile_w != 16) || (cfg->tile_h != 8 && cfg->tile_h != 16))
        return fail(XPR_ERR_INVALID, "tile size %dx%d not supported (8 or 16 each)", cfg->tile_w, cfg->tile_h);
    if (cfg->sh_degree < 0 || cfg->sh_degree > 3)
        return fail(XPR_ERR_INVALID, "sh_degree %d out of range [0, 3]", cfg->sh_degree);
    if (!(cfg->alpha_thresh > 0.f) || !(cfg->alpha_max <= 1.f) || !(cfg->alpha_thresh <= cfg->alpha_max))
        return fail(XPR_ERR_INVALID, "need 0 < alpha_thresh <= alpha_max <= 1");
    if (!(cfg->alpha_max < 1.f)) return fail(XPR_ERR_INVALID, "alpha_max must be < 1");
    if (!(cfg->t_eps >= 0.f)) return fail(XPR_ERR_INVALID, "t_eps must be >= 0");
    if (cfg->method != XPR_METHOD_3DGS && cfg->method != XPR_METHOD_3DGUT && cfg->method != XPR_METHOD_LINPRIM)
        return fail(XPR_ERR_INVALID, "method %d not supported (0 = 3DGS, 1 = 3DGUT, 2 = LinPrim)", cfg->method);
    if (cam->model == 1 && cfg->method != XPR_METHOD_3DGUT)
        return fail(XPR_ERR_INVALID, "the fisheye camera needs the 3DGUT method (the others linearise a pinhole)");
    for (int i = 0; i < 4; ++i)
        if (!(fabsf(cam->dist[i]) < 1e30f)) return fail(XPR_ERR_INVALID, "fisheye coefficient %d not finite", i);
    return XPR_OK;
}

// Projection and render entry points implement one method each.
int need_method(const XprConfig *cfg, int method, const char *fn) {
    if (cfg->method != method)
        return fail(XPR_ERR_INVALID, "%s implements method %d (%s) but cfg->method is %d", fn, method,
                    method == XPR_METHOD_3DGS ? "3DGS" : (method == XPR_METHOD_3DGUT ? "3DGUT" : "LinPrim"),
                    cfg->method);
    return XPR_OK;
}

static int check_n(int64_t n) {
    if (n < 0 || n > 0x7fffffffLL) return fail(XPR_ERR_INVALID, "primitive count %lld out of range", (long long)n);
    return XPR_OK;
}

int make_item_table(const XprCamera *cams, const XprItem *items, int n_items, const XprConfig &cfg, ItemTable &t,
                    int64_t *n_records, const char *fn) {
    if (n_items < 1 || n_items > kMaxItems)
        return fail(XPR_ERR_INVALID, "%s: item count %d out of range [1, %d]", fn, n_items, kMaxItems);
    if (!cams || !items) return fail(XPR_ERR_INVALID, "%s: NULL cameras or items", fn);
    memset(&t, 0, sizeof(t));
    t.count = n_items;
    int64_t rec = 0, tile = 0, pix = 0;
    for (int k = 0; k < n_items; ++k) {
        int s = validate_camera_config(cams + k, &cfg);
        if (s) return s;
        const XprItem &it = items[k];
        if (it.n < 0 || it.prim_offset < 0)
            return fail(XPR_ERR_INVALID, "%s: item %d has a negative primitive range", fn, k);
        if (it.rec_offset != rec || it.tile_offset != tile || it.pix_offset != pix)
            return fail(XPR_ERR_INVALID, "%s: item %d offsets (%lld, %lld, %lld) are not the running sums "
                        "(%lld, %lld, %lld)", fn, k, (long long)it.rec_offset, (long long)it.tile_offset,
                        (long long)it.pix_offset, (long long)rec, (long long)tile, (long long)pix);
        t.W[k] = cams[k].width;
        t.H[k] = cams[k].height;
        t.Wt[k] = tiles_x(cams[k], cfg);
        t.tile0[k] = tile;
        t.pix0[k] = pix;
        rec += (it.n + 31) / 32 * 32;
        tile += (int64_t)tiles_x(cams[k], cfg) * tiles_y(cams[k], cfg);
        pix += (int64_t)cams[k].width * cams[k].height;
    }
    t.tile0[n_items] = tile;
    if (rec > 0x7fffffffLL || tile > 0x7fffffffLL)
        return fail(XPR_ERR_INVALID, "%s: %lld records or %lld tiles exceed 2^31-1", fn, (long long)rec,
                    (long long)tile);
    if (n_records) *n_records = rec;
    return XPR_OK;
}

}  // namespace xpr

using namespace xpr;

extern "C" {

int xpr_version(void) { return 1; }

unsigned long long xpr_launch_count(void) { return g_launches.load(std::memory_order_relaxed); }

const char *xpr_last_error(void) { return g_err; }

int xpr_selftest_wait(uint32_t *zeroed, int32_t polls, void *stream) {
    if (!zeroed) return fail(XPR_ERR_INVALID, "xpr_selftest_wait: NULL buffer");
    if (polls < 1 || polls > (1 << 20)) return fail(XPR_ERR_INVALID, "xpr_selftest_wait: polls must be in [1, 2^20]");
    return lookback_selftest(zeroed, polls, as_stream(stream));
}

int xpr_device_check(void) {
    unsigned bits = 0;
    const int s = sort_device_errors(&bits);
    if (s != XPR_OK) return s;
    if (bits & 1u) return fail(XPR_ERR_TIMEOUT, "sort: a look-back wait gave up (flags %u)", bits);
    if (bits & 2u) return fail(XPR_ERR_INTERNAL, "sort: inconsistent chained-scan word or output position");
    return XPR_OK;
}

const char *xpr_status_string(int s) {
    switch (s) {
        case XPR_OK: return "ok";
        case XPR_ERR_INVALID: return "invalid argument";
        case XPR_ERR_CAPACITY: return "intersection capacity exceeded";
        case XPR_ERR_CUDA: return "CUDA error";
        case XPR_ERR_TIMEOUT: return "device wait timed out";
        case XPR_ERR_INTERNAL: return "internal consistency check failed";
        default: return "unknown status";
    }
}

int xpr_project(const XprPrims *prims, int64_t n, const XprCamera *cam, const XprConfig *cfg, float *rec,
                int32_t *bbox, int32_t *tile_count, int32_t *isect_count, void *stream) {
    int s = validate_camera_config(cam, cfg);
    if (s) return s;
    if ((s = need_method(cfg, XPR_METHOD_3DGS, "xpr_project"))) return s;
    if ((s = check_n(n))) return s;
    if (n == 0) return XPR_OK;
    if (!prims || !prims->mu || !prims->scale || !prims->quat || !prims->opacity || !rec || !bbox || !tile_count)
        return fail(XPR_ERR_INVALID, "xpr_project: NULL pointer");
    if (!aligned(prims->quat, 16) || !aligned(rec, 16) || !aligned(bbox, 16))
        return fail(XPR_ERR_INVALID, "xpr_project: quat, rec and bbox must be 16-byte aligned");
    return launch_project_fwd(*prims, n, *cam, *cfg, rec, bbox, tile_count, isect_count, as_stream(stream));
}

int xpr_project_host(const XprPrims *host, const XprPrims *dst, int64_t n, const XprCamera *cam,
                     const XprConfig *cfg, float *rec, int32_t *bbox, int32_t *tile_count, int32_t *isect_count,
                     void *stream) {
    int s = validate_camera_config(cam, cfg);
    if (s) return s;
    if ((s = need_method(cfg, XPR_METHOD_3DGS, "xpr_project_host"))) return s;
    if ((s = check_n(n))) return s;
    if (!host || !dst || !host->mu || !host->scale || !host->quat || !host->opacity || !dst->mu || !dst->scale ||
        !dst->quat || !dst->opacity || !rec || !bbox || !tile_count)
        return fail(XPR_ERR_INVALID, "xpr_project_host: NULL pointer");
    if (n == 0) return XPR_OK;
    if (!aligned(host->quat, 16) || !aligned(dst->quat, 16) || !aligned(rec, 16) || !aligned(bbox, 16))
        return fail(XPR_ERR_INVALID, "xpr_project_host: quat, rec and bbox must be 16-byte aligned");
    // the kernel dereferences the host arrays: each must be page-locked memory mapped for the device
    // (the kernel reads it at its device address)
    const float *hp[4] = {host->mu, host->scale, host->quat, host->opacity};
    const float *hd[4];
    for (int a = 0; a < 4; ++a) {
        cudaPointerAttributes at;
        if (cudaPointerGetAttributes(&at, hp[a]) != cudaSuccess) {
            cudaGetLastError();
            return fail(XPR_ERR_INVALID, "xpr_project_host: cannot query a host pointer");
        }
        if (at.type != cudaMemoryTypeHost || at.devicePointer == nullptr)
            return fail(XPR_ERR_INVALID, "xpr_project_host: host geometry must be page-locked and device-mapped");
        hd[a] = static_cast<const float *>(at.devicePointer);
    }
    if (!aligned(hd[2], 16)) return fail(XPR_ERR_INVALID, "xpr_project_host: quat must be 16-byte aligned");
    const XprPrims src = {hd[0], hd[1], hd[2], hd[3], dst->sh};
    const XprPrimsGrad copy = {const_cast<float *>(dst->mu), const_cast<float *>(dst->scale),
                               const_cast<float *>(dst->quat), const_cast<float *>(dst->opacity), nullptr};
    return launch_project_fwd(src, n, *cam, *cfg, rec, bbox, tile_count, isect_count, as_stream(stream), &copy);
}

size_t xpr_tile_bin_workspace(int64_t n) { return scan_partials_bytes(n < 0 ? 0 : n); }

}  // extern "C"

namespace xpr {
// n records; per_view > 0: records are view-major with per_view records per view and tile ids are
// offset by view * tiles-per-view.
int tile_bin_impl(const float *rec, const int32_t *bbox, const int32_t *tile_count, const int32_t *isect_count,
                  const int32_t *order, int64_t n, const XprCamera *cam, const XprConfig *cfg, int32_t *offsets,
                  uint64_t *keys, uint32_t *tiles, uint32_t *vals, int64_t capacity, int64_t *n_isect,
                  void *workspace, size_t ws_bytes, void *stream, int64_t per_view, const float *lp_sd = nullptr) {
    int s = validate_camera_config(cam, cfg);
    if (s) return s;
    // LinPrim culls from its shader data (xpr_tile_bin_lp); the other methods from the records
    if ((cfg->method == XPR_METHOD_LINPRIM) != (lp_sd != nullptr))
        return fail(XPR_ERR_INVALID, lp_sd ? "xpr_tile_bin_lp needs cfg->method == LinPrim"
                                           : "xpr_tile_bin: LinPrim binning is xpr_tile_bin_lp (it needs sd)");
    if (lp_sd && n > 0 && !aligned(lp_sd, 16)) return fail(XPR_ERR_INVALID, "xpr_tile_bin_lp: sd must be 16-byte aligned");
    if ((s = check_n(n))) return s;
    if (!offsets || !n_isect || (n > 0 && (!rec || !bbox || !tile_count || !workspace)))
        return fail(XPR_ERR_INVALID, "xpr_tile_bin: NULL pointer");
    if (capacity < 0) return fail(XPR_ERR_INVALID, "xpr_tile_bin: negative capacity");
    if (n > 0 && (!aligned(rec, 16) || !aligned(bbox, 16) || !aligned(workspace, 256)))
        return fail(XPR_ERR_INVALID, "xpr_tile_bin: rec/bbox must be 16-byte and workspace 256-byte aligned");
    if (ws_bytes < xpr_tile_bin_workspace(n))
        return fail(XPR_ERR_INVALID, "xpr_tile_bin: workspace %zu < %zu bytes", ws_bytes, xpr_tile_bin_workspace(n));
    cudaStream_t st = as_stream(stream);
    if (n == 0) {
        XPR_CUDA_TRY(cudaMemsetAsync(offsets, 0, sizeof(int32_t), st));
        *n_isect = 0;
        return XPR_OK;
    }
    if (isect_count) {
        // per-primitive counts from xpr_project, taken in emission order
        if ((s = launch_exclusive_scan(isect_count, offsets, n, workspace, nullptr, st, order))) return s;
    } else {
        if (lp_sd) {
            if ((s = launch_lp_bin_count(lp_sd, bbox, tile_count, order, n, *cam, *cfg, offsets, st))) return s;
        } else {
            if ((s = launch_bin_count(rec, bbox, tile_count, order, n, *cam, *cfg, offsets, st))) return s;
        }
        if ((s = launch_exclusive_scan(offsets, offsets, n, workspace, nullptr, st))) return s;
    }
    const int64_t *tot_dev = scan_total_ptr(workspace, n);
    int64_t total = 0;
    XPR_CUDA_TRY(cudaMemcpyAsync(&total, tot_dev, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    XPR_CUDA_TRY(cudaStreamSynchronize(st));
    *n_isect = total;
    if (total > 0x7fffffffLL) return fail(XPR_ERR_CAPACITY, "xpr_tile_bin: %lld intersections exceed 2^31-1",
                                          (long long)total);
    if (total > capacity)
        return fail(XPR_ERR_CAPACITY, "xpr_tile_bin: %lld intersections > capacity %lld", (long long)total,
                    (long long)capacity);
    if (total > 0 && ((!keys && !tiles) || !vals)) return fail(XPR_ERR_INVALID, "xpr_tile_bin: NULL keys/tiles/vals");
    if (lp_sd)
        return launch_lp_bin_emit(rec, lp_sd, bbox, tile_count, order, n, *cam, *cfg, offsets, keys, tiles, vals, st,
                                  per_view);
    return launch_bin_emit(rec, bbox, tile_count, order, n, *cam, *cfg, offsets, keys, tiles, vals, st, per_view);
}
}  // namespace xpr

extern "C" {

int xpr_tile_bin(const float *rec, const int32_t *bbox, const int32_t *tile_count, const int32_t *isect_count,
                 const int32_t *order, int64_t n, const XprCamera *cam, const XprConfig *cfg, int32_t *offsets,
                 uint64_t *keys, uint32_t *tiles, uint32_t *vals, int64_t capacity, int64_t *n_isect,
                 void *workspace, size_t ws_bytes, void *stream) {
    return tile_bin_impl(rec, bbox, tile_count, isect_count, order, n, cam, cfg, offsets, keys, tiles, vals,
                         capacity, n_isect, workspace, ws_bytes, stream, 0);
}

size_t xpr_sort_tiles_workspace(int64_t n_isect, int32_t n_tiles) {
    return sort_tiles_workspace_bytes(n_isect < 0 ? 0 : n_isect, n_tiles);
}

int xpr_sort_tiles(const uint32_t *tiles_in, const uint32_t *vals_in, int64_t n_isect, int32_t n_tiles,
                   uint32_t *tiles_out, uint32_t *vals_out, int32_t *ranges, void *workspace, size_t ws_bytes,
                   void *stream) {
    if (n_isect < 0 || n_isect > 0x7fffffffLL) return fail(XPR_ERR_INVALID, "xpr_sort_tiles: bad count");
    if (n_tiles < 1) return fail(XPR_ERR_INVALID, "xpr_sort_tiles: n_tiles must be >= 1");
    if (!ranges) return fail(XPR_ERR_INVALID, "xpr_sort_tiles: NULL ranges");
    if (n_isect > 0 && (!tiles_in || !vals_in || !vals_out || !workspace))
        return fail(XPR_ERR_INVALID, "xpr_sort_tiles: NULL pointer");
    if (n_isect > 0 && (tiles_in == tiles_out || vals_in == vals_out))
        return fail(XPR_ERR_INVALID, "xpr_sort_tiles: input and output buffers must not alias");
    if (n_isect > 0 && !aligned(workspace, 256)) return fail(XPR_ERR_INVALID, "xpr_sort_tiles: workspace alignment");
    return launch_sort_tiles(tiles_in, vals_in, n_isect, n_tiles, tiles_out, vals_out, ranges, workspace, ws_bytes,
                             as_stream(stream));
}

size_t xpr_depth_order_workspace(int64_t n) { return depth_order_workspace_bytes(n < 0 ? 0 : n); }

int xpr_depth_order(const float *rec, const int32_t *tile_count, int64_t n, int32_t *order, void *workspace,
                    size_t ws_bytes, void *stream) {
    int s = check_n(n);
    if (s) return s;
    if (n == 0) return XPR_OK;
    if (!rec || !tile_count || !order || !workspace) return fail(XPR_ERR_INVALID, "xpr_depth_order: NULL pointer");
    if (!aligned(workspace, 256)) return fail(XPR_ERR_INVALID, "xpr_depth_order: workspace must be 256-byte aligned");
    return launch_depth_order(rec, tile_count, n, order, workspace, ws_bytes, as_stream(stream));
}

size_t xpr_sort_workspace(int64_t n_isect, int32_t n_tiles) {
    return sort_workspace_bytes(n_isect < 0 ? 0 : n_isect, n_tiles);
}

int xpr_sort(const uint64_t *keys_in, const uint32_t *vals_in, int64_t n_isect, int32_t n_tiles, int32_t begin_bit,
             uint64_t *keys_out, uint32_t *vals_out, int32_t *ranges, void *workspace, size_t ws_bytes,
             void *stream) {
    if (n_isect < 0 || n_isect > 0x7fffffffLL) return fail(XPR_ERR_INVALID, "xpr_sort: bad count");
    if (n_tiles < 1) return fail(XPR_ERR_INVALID, "xpr_sort: n_tiles must be >= 1");
    if (begin_bit < 0 || begin_bit > 32) return fail(XPR_ERR_INVALID, "xpr_sort: begin_bit must be in [0, 32]");
    if (!ranges) return fail(XPR_ERR_INVALID, "xpr_sort: NULL ranges");
    if (n_isect > 0 && (!keys_in || !vals_in || !keys_out || !vals_out || !workspace))
        return fail(XPR_ERR_INVALID, "xpr_sort: NULL pointer");
    if (n_isect > 0 && (keys_in == keys_out || vals_in == vals_out))
        return fail(XPR_ERR_INVALID, "xpr_sort: input and output buffers must not alias");
    if (n_isect > 0 && !aligned(workspace, 256)) return fail(XPR_ERR_INVALID, "xpr_sort: workspace alignment");
    return launch_sort(keys_in, vals_in, n_isect, n_tiles, begin_bit, keys_out, vals_out, ranges, workspace,
                       ws_bytes, as_stream(stream));
}

int xpr_render_fwd(const float *rec, int64_t n, const uint32_t *vals, const int32_t *ranges, const XprCamera *cam,
                   const XprConfig *cfg, float *image, float *t_final, int32_t *n_contrib, void *stream) {
    int s = validate_camera_config(cam, cfg);
    if (s) return s;
    if ((s = need_method(cfg, XPR_METHOD_3DGS, "xpr_render_fwd"))) return s;
    if ((s = check_n(n))) return s;
    if (!ranges || !image || !t_final || !n_contrib) return fail(XPR_ERR_INVALID, "xpr_render_fwd: NULL pointer");
    if (n > 0 && (!rec || !aligned(rec, 16))) return fail(XPR_ERR_INVALID, "xpr_render_fwd: rec NULL or unaligned");
    if (!aligned(ranges, 8)) return fail(XPR_ERR_INVALID, "xpr_render_fwd: ranges must be 8-byte aligned");
    return launch_render_fwd(rec, n, vals, ranges, *cam, *cfg, image, t_final, n_contrib, as_stream(stream));
}

int xpr_project_bwd(const XprPrims *prims, int64_t n, const XprCamera *cam, const XprConfig *cfg,
                    const float *d_rec, const XprPrimsGrad *d_prims, void *stream) {
    int s = validate_camera_config(cam, cfg);
    if (s) return s;
    if ((s = need_method(cfg, XPR_METHOD_3DGS, "xpr_project_bwd"))) return s;
    if ((s = check_n(n))) return s;
    if (n == 0) return XPR_OK;
    if (!prims || !d_prims || !d_rec || !prims->mu || !prims->scale || !prims->quat || !prims->opacity ||
        !prims->sh || !d_prims->mu || !d_prims->scale || !d_prims->quat || !d_prims->opacity || !d_prims->sh)
        return fail(XPR_ERR_INVALID, "xpr_project_bwd: NULL pointer");
    if (!aligned(prims->quat, 16) || !aligned(d_prims->quat, 16) || !aligned(d_rec, 16))
        return fail(XPR_ERR_INVALID, "xpr_project_bwd: quat and d_rec must be 16-byte aligned");
    return launch_project_bwd(*prims, n, *cam, *cfg, d_rec, *d_prims, as_stream(stream));
}

int xpr_render_bwd(const float *rec, int64_t n, const uint32_t *vals, const int32_t *ranges, const XprCamera *cam,
                   const XprConfig *cfg, const float *t_final, const int32_t *n_contrib, const float *d_image,
                   float *d_rec, const XprPrims *prims, const XprPrimsGrad *d_prims, void *stream) {
    int s = validate_camera_config(cam, cfg);
    if (s) return s;
    if ((s = need_method(cfg, XPR_METHOD_3DGS, "xpr_render_bwd"))) return s;
    if ((s = check_n(n))) return s;
    if (!ranges || !t_final || !n_contrib || !d_image) return fail(XPR_ERR_INVALID, "xpr_render_bwd: NULL pointer");
    if (n == 0) return XPR_OK;
    if (!rec || !d_rec || !aligned(rec, 16) || !aligned(d_rec, 16))
        return fail(XPR_ERR_INVALID, "xpr_render_bwd: rec/d_rec NULL or not 16-byte aligned");
    cudaStream_t st = as_stream(stream);
    if ((s = launch_render_bwd(rec, vals, ranges, *cam, *cfg, t_final, n_contrib, d_image, d_rec, n, st))) return s;
    if (prims && d_prims) return xpr_project_bwd(prims, n, cam, cfg, d_rec, d_prims, stream);
    return XPR_OK;
}

// ---- multi-view (batched) form ------------------------------------------------------------

static int check_views(int32_t n_views, int64_t n) {
    if (n_views < 1 || n_views > kMaxViews)
        return fail(XPR_ERR_INVALID, "view count %d out of range [1, %d]", n_views, kMaxViews);
    if (n < 0 || n * (int64_t)n_views > 0x7fffffffLL)
        return fail(XPR_ERR_INVALID, "views x primitives = %lld x %d exceeds 2^31-1 records", (long long)n, n_views);
    return XPR_OK;
}

int xpr_project_views(const XprPrims *prims, int64_t n, const XprCamera *cams, int32_t n_views, const XprConfig *cfg,
                      float *rec, int32_t *bbox, int32_t *tile_count, int32_t *isect_count, void *stream) {
    int s = check_views(n_views, n);
    if (s) return s;
    if (!cams) return fail(XPR_ERR_INVALID, "xpr_project_views: NULL cameras");
    for (int v = 0; v < n_views; ++v)
        if ((s = validate_camera_config(cams + v, cfg))) return s;
    if ((s = need_method(cfg, XPR_METHOD_3DGS, "xpr_project_views"))) return s;
    if (n == 0) return XPR_OK;
    if (!prims || !prims->mu || !prims->scale || !prims->quat || !prims->opacity || !rec || !bbox || !tile_count)
        return fail(XPR_ERR_INVALID, "xpr_project_views: NULL pointer");
    if (!aligned(prims->quat, 16) || !aligned(rec, 16) || !aligned(bbox, 16))
        return fail(XPR_ERR_INVALID, "xpr_project_views: quat, rec and bbox must be 16-byte aligned");
    return launch_project_fwd_views(*prims, n, cams, n_views, *cfg, rec, bbox, tile_count, isect_count,
                                    as_stream(stream));
}

int xpr_depth_order_views(const float *rec, const int32_t *tile_count, int64_t n, int32_t n_views, int32_t *order,
                          void *workspace, size_t ws_bytes, void *stream) {
    int s = check_views(n_views, n);
    if (s) return s;
    if (n == 0) return XPR_OK;
    if (!rec || !tile_count || !order || !workspace) return fail(XPR_ERR_INVALID, "xpr_depth_order_views: NULL");
    if (!aligned(workspace, 256)) return fail(XPR_ERR_INVALID, "xpr_depth_order_views: workspace alignment");
    return launch_depth_order(rec, tile_count, n * n_views, order, workspace, ws_bytes, as_stream(stream), n,
                              n_views);
}

int xpr_tile_bin_views(const float *rec, const int32_t *bbox, const int32_t *tile_count, const int32_t *isect_count,
                       const int32_t *order, int64_t n, int32_t n_views, const XprCamera *cam, const XprConfig *cfg,
                       int32_t *offsets, uint32_t *tiles, uint32_t *vals, int64_t capacity, int64_t *n_isect,
                       void *workspace, size_t ws_bytes, void *stream) {
    int s = check_views(n_views, n);
    if (s) return s;
    return tile_bin_impl(rec, bbox, tile_count, isect_count, order, n * n_views, cam, cfg, offsets, nullptr, tiles,
                         vals, capacity, n_isect, workspace, ws_bytes, stream, n);
}

size_t xpr_tile_worklist_workspace(int32_t n_tiles) { return worklist_workspace_bytes(n_tiles < 0 ? 0 : n_tiles); }

int xpr_tile_worklist(const int32_t *ranges, int32_t n_tiles, int32_t *worklist, void *workspace, size_t ws_bytes,
                      void *stream) {
    if (n_tiles < 0) return fail(XPR_ERR_INVALID, "xpr_tile_worklist: negative tile count");
    if (n_tiles == 0) return XPR_OK;
    if (!ranges || !worklist || !workspace) return fail(XPR_ERR_INVALID, "xpr_tile_worklist: NULL pointer");
    if (!aligned(ranges, 8) || !aligned(workspace, 256))
        return fail(XPR_ERR_INVALID, "xpr_tile_worklist: ranges/workspace alignment");
    return launch_tile_worklist(ranges, n_tiles, worklist, workspace, ws_bytes, as_stream(stream));
}

int xpr_render_fwd_views(const float *rec, int64_t n, int32_t n_views, const uint32_t *vals, const int32_t *ranges,
                         const XprCamera *cam, const XprConfig *cfg, float *image, float *t_final, int32_t *n_contrib,
                         const int32_t *worklist, int32_t *counter, void *stream) {
    int s = validate_camera_config(cam, cfg);
    if (s) return s;
    if ((s = need_method(cfg, XPR_METHOD_3DGS, "xpr_render_fwd_views"))) return s;
    if ((s = check_views(n_views, n))) return s;
    if (!ranges || !image || !t_final || !n_contrib) return fail(XPR_ERR_INVALID, "xpr_render_fwd_views: NULL");
    if (n > 0 && (!rec || !aligned(rec, 16))) return fail(XPR_ERR_INVALID, "xpr_render_fwd_views: rec");
    if (worklist && !counter) return fail(XPR_ERR_INVALID, "xpr_render_fwd_views: worklist needs a counter");
    if (!aligned(ranges, 8)) return fail(XPR_ERR_INVALID, "xpr_render_fwd_views: ranges must be 8-byte aligned");
    return launch_render_fwd_views(rec, n * n_views, vals, ranges, n_views, *cam, *cfg, image, t_final, n_contrib,
                                   worklist, counter, as_stream(stream));
}

int xpr_render_bwd_views(const float *rec, int64_t n, int32_t n_views, const uint32_t *vals, const int32_t *ranges,
                         const XprCamera *cam, const XprConfig *cfg, const float *t_final, const int32_t *n_contrib,
                         const float *d_image, float *d_rec, const int32_t *worklist, int32_t *counter,
                         void *stream) {
    int s = validate_camera_config(cam, cfg);
    if (s) return s;
    if ((s = need_method(cfg, XPR_METHOD_3DGS, "xpr_render_bwd_views"))) return s;
    if ((s = check_views(n_views, n))) return s;
    if (!ranges || !t_final || !n_contrib || !d_image) return fail(XPR_ERR_INVALID, "xpr_render_bwd_views: NULL");
    if (n == 0) return XPR_OK;
    if (!rec || !d_rec || !aligned(rec, 16) || !aligned(d_rec, 16))
        return fail(XPR_ERR_INVALID, "xpr_render_bwd_views: rec/d_rec NULL or not 16-byte aligned");
    if (worklist && !counter) return fail(XPR_ERR_INVALID, "xpr_render_bwd_views: worklist needs a counter");
    return launch_render_bwd_views(rec, vals, ranges, n_views, *cam, *cfg, t_final, n_contrib, d_image, d_rec,
                                   n * n_views, worklist, counter, as_stream(stream));
}

int xpr_project_bwd_views(const XprPrims *prims, int64_t n, const XprCamera *cams, int32_t n_views,
                          const XprConfig *cfg, const float *d_rec, const XprPrimsGrad *d_prims, void *stream) {
    int s = check_views(n_views, n);
    if (s) return s;
    if (!cams) return fail(XPR_ERR_INVALID, "xpr_project_bwd_views: NULL cameras");
    for (int v = 0; v < n_views; ++v)
        if ((s = validate_camera_config(cams + v, cfg))) return s;
    if ((s = need_method(cfg, XPR_METHOD_3DGS, "xpr_project_bwd_views"))) return s;
    if (n == 0) return XPR_OK;
    if (!prims || !d_prims || !d_rec || !prims->mu || !prims->scale || !prims->quat || !prims->opacity ||
        !prims->sh || !d_prims->mu || !d_prims->scale || !d_prims->quat || !d_prims->opacity || !d_prims->sh)
        return fail(XPR_ERR_INVALID, "xpr_project_bwd_views: NULL pointer");
    if (!aligned(prims->quat, 16) || !aligned(d_prims->quat, 16) || !aligned(d_rec, 16))
        return fail(XPR_ERR_INVALID, "xpr_project_bwd_views: quat and d_rec must be 16-byte aligned");
    return launch_project_bwd_views(*prims, n, cams, n_views, *cfg, d_rec, *d_prims, as_stream(stream));
}

// ---- multi-scene batched form (items) ------------------------------------------------------


int xpr_project_items(const XprPrims *prims, const XprCamera *cams, const XprItem *items, int32_t n_items,
                      const XprConfig *cfg, float *rec, int32_t *bbox, int32_t *tile_count, void *stream) {
    if (!cfg) return fail(XPR_ERR_INVALID, "xpr_project_items: NULL config");
    ItemTable t;
    int64_t R = 0;
    int s = make_item_table(cams, items, n_items, *cfg, t, &R, "xpr_project_items");
    if (s) return s;
    if ((s = need_method(cfg, XPR_METHOD_3DGS, "xpr_project_items"))) return s;
    if (R == 0) return XPR_OK;
    if (!prims || !prims->mu || !prims->scale || !prims->quat || !prims->opacity || !prims->sh || !rec || !bbox ||
        !tile_count)
        return fail(XPR_ERR_INVALID, "xpr_project_items: NULL pointer");
    if (!aligned(prims->quat, 16) || !aligned(rec, 16) || !aligned(bbox, 16))
        return fail(XPR_ERR_INVALID, "xpr_project_items: quat, rec and bbox must be 16-byte aligned");
    return launch_project_items(*prims, cams, items, n_items, *cfg, rec, bbox, tile_count, as_stream(stream));
}

int xpr_depth_order_items(const float *rec, const int32_t *tile_count, const XprItem *items, int32_t n_items,
                          int32_t *order, void *workspace, size_t ws_bytes, void *stream) {
    if (n_items < 1 || n_items > kMaxItems || !items)
        return fail(XPR_ERR_INVALID, "xpr_depth_order_items: item count %d out of range [1, %d]", n_items, kMaxItems);
    int64_t rec_end = 0;
    for (int k = 0; k < n_items; ++k) {
        if (items[k].n < 0 || items[k].rec_offset != rec_end)
            return fail(XPR_ERR_INVALID, "xpr_depth_order_items: item %d record block is not the running sum", k);
        rec_end += (items[k].n + 31) / 32 * 32;
    }
    if (rec_end == 0) return XPR_OK;
    if (rec_end > 0x7fffffffLL) return fail(XPR_ERR_INVALID, "xpr_depth_order_items: too many records");
    if (!rec || !tile_count || !order || !workspace) return fail(XPR_ERR_INVALID, "xpr_depth_order_items: NULL");
    if (!aligned(workspace, 256)) return fail(XPR_ERR_INVALID, "xpr_depth_order_items: workspace alignment");
    return launch_depth_order_items(rec, tile_count, items, n_items, order, workspace, ws_bytes, as_stream(stream));
}

size_t xpr_bin_sorted_items_workspace(const XprCamera *cams, const XprItem *items, int32_t n_items,
                                      const XprConfig *cfg) {
    ItemTable t;
    if (!cfg || make_item_table(cams, items, n_items, *cfg, t, nullptr, "xpr_bin_sorted_items_workspace") != XPR_OK)
        return 0;
    return binsort_items_workspace_bytes(cams, items, n_items, *cfg);
}

int xpr_bin_sorted_items(const float *rec, const int32_t *bbox, const int32_t *tile_count, const int32_t *order,
                         const XprCamera *cams, const XprItem *items, int32_t n_items, const XprConfig *cfg,
                         int32_t *ranges, uint32_t *vals, int64_t capacity, int64_t *n_isect, void *workspace,
                         size_t ws_bytes, void *stream) {
    if (!cfg) return fail(XPR_ERR_INVALID, "xpr_bin_sorted_items: NULL config");
    ItemTable t;
    int64_t R = 0;
    int s = make_item_table(cams, items, n_items, *cfg, t, &R, "xpr_bin_sorted_items");
    if (s) return s;
    if ((s = need_method(cfg, XPR_METHOD_3DGS, "xpr_bin_sorted_items"))) return s;
    if (!binsort_items_supported(cams, n_items, *cfg))
        return fail(XPR_ERR_INVALID, "xpr_bin_sorted_items: a camera has more than 4096 tile columns");
    if (!ranges || !n_isect) return fail(XPR_ERR_INVALID, "xpr_bin_sorted_items: NULL ranges or n_isect");
    if (capacity < 0) return fail(XPR_ERR_INVALID, "xpr_bin_sorted_items: negative capacity");
    if (R > 0 && (!rec || !bbox || !tile_count || !order || !workspace))
        return fail(XPR_ERR_INVALID, "xpr_bin_sorted_items: NULL pointer");
    if (R > 0 && (!aligned(rec, 16) || !aligned(bbox, 16) || !aligned(workspace, 256)))
        return fail(XPR_ERR_INVALID, "xpr_bin_sorted_items: rec/bbox 16-byte and workspace 256-byte alignment");
    return launch_binsort_items(rec, bbox, tile_count, order, cams, items, n_items, *cfg, ranges, vals, capacity,
                                n_isect, workspace, ws_bytes, as_stream(stream));
}

int xpr_render_fwd_items(const float *rec, const uint32_t *vals, const int32_t *ranges, const XprCamera *cams,
                         const XprItem *items, int32_t n_items, const XprConfig *cfg, float *image, float *t_final,
                         int32_t *n_contrib, const int32_t *worklist, int32_t *counter, void *stream) {
    if (!cfg) return fail(XPR_ERR_INVALID, "xpr_render_fwd_items: NULL config");
    ItemTable t;
    int64_t R = 0;
    int s = make_item_table(cams, items, n_items, *cfg, t, &R, "xpr_render_fwd_items");
    if (s) return s;
    if ((s = need_method(cfg, XPR_METHOD_3DGS, "xpr_render_fwd_items"))) return s;
    if (!ranges || !image || !t_final || !n_contrib) return fail(XPR_ERR_INVALID, "xpr_render_fwd_items: NULL");
    if (R > 0 && (!rec || !aligned(rec, 16))) return fail(XPR_ERR_INVALID, "xpr_render_fwd_items: rec");
    if (worklist && !counter) return fail(XPR_ERR_INVALID, "xpr_render_fwd_items: worklist needs a counter");
    if (!aligned(ranges, 8)) return fail(XPR_ERR_INVALID, "xpr_render_fwd_items: ranges must be 8-byte aligned");
    return launch_render_fwd_items(rec, R, vals, ranges, t, *cfg, image, t_final, n_contrib, worklist, counter,
                                   as_stream(stream));
}

int xpr_render_bwd_items(const float *rec, const uint32_t *vals, const int32_t *ranges, const XprCamera *cams,
                         const XprItem *items, int32_t n_items, const XprConfig *cfg, const float *t_final,
                         const int32_t *n_contrib, const float *d_image, float *d_rec, const int32_t *worklist,
                         int32_t *counter, void *stream) {
    if (!cfg) return fail(XPR_ERR_INVALID, "xpr_render_bwd_items: NULL config");
    ItemTable t;
    int64_t R = 0;
    int s = make_item_table(cams, items, n_items, *cfg, t, &R, "xpr_render_bwd_items");
    if (s) return s;
    if ((s = need_method(cfg, XPR_METHOD_3DGS, "xpr_render_bwd_items"))) return s;
    if (!ranges || !t_final || !n_contrib || !d_image) return fail(XPR_ERR_INVALID, "xpr_render_bwd_items: NULL");
    if (R == 0) return XPR_OK;
    if (!rec || !d_rec || !aligned(rec, 16) || !aligned(d_rec, 16))
        return fail(XPR_ERR_INVALID, "xpr_render_bwd_items: rec/d_rec NULL or not 16-byte aligned");
    if (worklist && !counter) return fail(XPR_ERR_INVALID, "xpr_render_bwd_items: worklist needs a counter");
    return launch_render_bwd_items(rec, R, vals, ranges, t, *cfg, t_final, n_contrib, d_image, d_rec, worklist,
                                   counter, as_stream(stream));
}

int xpr_project_bwd_items(const XprPrims *prims, int64_t n_prims, const XprCamera *cams, const XprItem *items,
                          int32_t n_items, const XprConfig *cfg, const float *d_rec, const XprPrimsGrad *d_prims,
                          void *stream) {
    if (!cfg) return fail(XPR_ERR_INVALID, "xpr_project_bwd_items: NULL config");
    ItemTable t;
    int64_t R = 0;
    int s = make_item_table(cams, items, n_items, *cfg, t, &R, "xpr_project_bwd_items");
    if (s) return s;
    if ((s = need_method(cfg, XPR_METHOD_3DGS, "xpr_project_bwd_items"))) return s;
    for (int k = 0; k < n_items; ++k)
        if (items[k].prim_offset + items[k].n > n_prims)
            return fail(XPR_ERR_INVALID, "xpr_project_bwd_items: item %d reaches past the %lld primitives", k,
                        (long long)n_prims);
    if (n_prims == 0) return XPR_OK;
    if (!prims || !d_prims || !prims->mu || !prims->scale || !prims->quat || !prims->opacity || !prims->sh ||
        !d_prims->mu || !d_prims->scale || !d_prims->quat || !d_prims->opacity || !d_prims->sh || (R > 0 && !d_rec))
        return fail(XPR_ERR_INVALID, "xpr_project_bwd_items: NULL pointer");
    if (!aligned(prims->quat, 16) || !aligned(d_prims->quat, 16) || (d_rec && !aligned(d_rec, 16)))
        return fail(XPR_ERR_INVALID, "xpr_project_bwd_items: quat and d_rec must be 16-byte aligned");
    return launch_project_bwd_items(*prims, n_prims, cams, items, n_items, *cfg, d_rec, *d_prims, as_stream(stream));
}

// Workspace layout of xpr_forward_items (every part 256-byte aligned).  The binning's scratch is
// one region: the rows binning's workspace with room for cap / 2 + R span slots (the spans hold
// from about three to nine pairs each on the serving workloads), else, or when the spans outgrow
// that room, the key path's offsets, scan partials, tile ids, values and sort scratch.
struct FwdItemsWs {
    size_t rec, bbox, tc, isect, order, depth, vals, ranges, worklist, wl_ws, counter, bin, total;
    size_t bin_bytes;
    size_t k_offsets, k_scan, k_tiles, k_vals_in, k_sort;  // the key path, inside the bin region
};

static size_t up256(size_t b) { return (b + 255) / 256 * 256; }

static FwdItemsWs fwd_items_layout(int64_t R, int64_t S, int64_t capacity, const RowItems *rows) {
    const size_t cap = (size_t)std::max<int64_t>(capacity, 1);
    FwdItemsWs w;
    size_t o = 0;
    auto take = [&](size_t &field, size_t bytes) {
        field = o;
        o += up256(bytes);
    };
    take(w.rec, (size_t)R * XPR_REC_FLOATS * 4);
    take(w.bbox, (size_t)R * 16);
    take(w.tc, (size_t)R * 4);
    take(w.isect, (size_t)R * 4);
    take(w.order, (size_t)R * 4);
    take(w.depth, depth_order_workspace_bytes(R));
    take(w.vals, cap * 4);
    take(w.ranges, (size_t)S * 8);
    take(w.worklist, (size_t)S * 4);
    take(w.wl_ws, worklist_workspace_bytes((int32_t)S));
    take(w.counter, 256);
    size_t k = 0;
    w.k_offsets = k;
    k += up256(((size_t)R + 1) * 4);
    w.k_scan = k;
    k += up256(scan_partials_bytes(R));
    w.k_tiles = k;
    k += up256(cap * 4);
    w.k_vals_in = k;
    k += up256(cap * 4);
    w.k_sort = k;
    k += up256(sort_tiles_workspace_bytes((int64_t)cap, (int32_t)S));
    if (rows) k = std::max(k, bin_rows_workspace_bytes(R, (int64_t)cap / 2 + R, (int64_t)cap, *rows));
    w.bin_bytes = k;
    take(w.bin, k);
    w.total = o;
    return w;
}

size_t xpr_forward_items_workspace(const XprCamera *cams, const XprItem *items, int32_t n_items, const XprConfig *cfg,
                                   int64_t capacity) {
    ItemTable t;
    int64_t R = 0;
    if (!cfg || capacity < 0 || capacity > 0x7fffffffLL ||
        make_item_table(cams, items, n_items, *cfg, t, &R, "xpr_forward_items_workspace") != XPR_OK)
        return 0;
    const RowItems rt = row_items_items(cams, items, n_items, *cfg);
    return fwd_items_layout(R, t.tile0[n_items], capacity, bin_rows_supported(rt) ? &rt : nullptr).total;
}

int xpr_forward_items(const XprPrims *prims, const XprCamera *cams, const XprItem *items, int32_t n_items,
                      const XprConfig *cfg, float *image, float *t_final, int32_t *n_contrib, int64_t capacity,
                      int64_t *n_isect, void *workspace, size_t ws_bytes, void *stream) {
    if (!cfg) return fail(XPR_ERR_INVALID, "xpr_forward_items: NULL config");
    ItemTable t;
    int64_t R = 0;
    int s = make_item_table(cams, items, n_items, *cfg, t, &R, "xpr_forward_items");
    if (s) return s;
    if ((s = need_method(cfg, XPR_METHOD_3DGS, "xpr_forward_items"))) return s;
    if (!n_isect || capacity < 0 || capacity > 0x7fffffffLL)
        return fail(XPR_ERR_INVALID, "xpr_forward_items: NULL n_isect or capacity out of range");
    const int64_t S = t.tile0[n_items];
    if (!image || !t_final || !n_contrib || !workspace)
        return fail(XPR_ERR_INVALID, "xpr_forward_items: NULL output or workspace");
    if (R > 0 && (!prims || !prims->mu || !prims->scale || !prims->quat || !prims->opacity || !prims->sh))
        return fail(XPR_ERR_INVALID, "xpr_forward_items: NULL primitive array");
    if (R > 0 && !aligned(prims->quat, 16)) return fail(XPR_ERR_INVALID, "xpr_forward_items: quat alignment");
    if (!aligned(workspace, 256)) return fail(XPR_ERR_INVALID, "xpr_forward_items: workspace must be 256-byte aligned");
    const RowItems rt = row_items_items(cams, items, n_items, *cfg);
    const bool by_rows = bin_rows_supported(rt);
    const FwdItemsWs L = fwd_items_layout(R, S, capacity, by_rows ? &rt : nullptr);
    if (ws_bytes < L.total)
        return fail(XPR_ERR_INVALID, "xpr_forward_items: workspace %zu < %zu bytes", ws_bytes, L.total);
    char *w = reinterpret_cast<char *>(workspace);
    float *rec = reinterpret_cast<float *>(w + L.rec);
    int32_t *bbox = reinterpret_cast<int32_t *>(w + L.bbox);
    int32_t *tc = reinterpret_cast<int32_t *>(w + L.tc);
    int32_t *isect = reinterpret_cast<int32_t *>(w + L.isect);
    int32_t *order = reinterpret_cast<int32_t *>(w + L.order);
    uint32_t *vals = reinterpret_cast<uint32_t *>(w + L.vals);
    int32_t *ranges = reinterpret_cast<int32_t *>(w + L.ranges);
    int32_t *wl = reinterpret_cast<int32_t *>(w + L.worklist);
    int32_t *counter = reinterpret_cast<int32_t *>(w + L.counter);
    char *bin = w + L.bin;
    cudaStream_t st = as_stream(stream);
    *n_isect = 0;
    int64_t total = 0;
    bool binned = false;
    if (R > 0) {
        // projection (with the exact kept-tile counts for the key path; the rows binning finds the
        // pair total in its span scan), depth order per item
        if ((s = launch_project_items(*prims, cams, items, n_items, *cfg, rec, bbox, tc, st,
                                      by_rows ? nullptr : isect)))
            return s;
        if ((s = launch_depth_order_items(rec, tc, items, n_items, order, w + L.depth,
                                          depth_order_workspace_bytes(R), st)))
            return s;
    }
    if (R > 0 && by_rows) {
        // binning and tile sort by rows (synchronises for the span total, then for the pair total)
        int64_t spans = 0;
        s = launch_bin_rows(rec, bbox, tc, nullptr, order, R, rt, *cfg, ranges, vals, capacity, &total, &spans, bin,
                            L.bin_bytes, st);
        *n_isect = total;
        if (s == XPR_OK) binned = true;
        else if (s != XPR_ERR_CAPACITY) return s;
        else if (total > capacity)
            return fail(XPR_ERR_CAPACITY, "xpr_forward_items: %lld intersections > capacity %lld", (long long)total,
                        (long long)capacity);
        // else the spans outgrew their room: the key path below gives the same lists, from the
        // kept-tile counts (the projection again, now with them: the same records)
        else if ((s = launch_project_items(*prims, cams, items, n_items, *cfg, rec, bbox, tc, st, isect)))
            return s;
    }
    if (!binned) {
        int32_t *offsets = reinterpret_cast<int32_t *>(bin + L.k_offsets);
        uint32_t *tiles = reinterpret_cast<uint32_t *>(bin + L.k_tiles);
        uint32_t *vals_in = reinterpret_cast<uint32_t *>(bin + L.k_vals_in);
        total = 0;
        if (R > 0) {
            if ((s = launch_exclusive_scan(isect, offsets, R, bin + L.k_scan, nullptr, st, order))) return s;
            XPR_CUDA_TRY(cudaMemcpyAsync(&total, scan_total_ptr(bin + L.k_scan, R), sizeof(int64_t),
                                         cudaMemcpyDeviceToHost, st));
            XPR_CUDA_TRY(cudaStreamSynchronize(st));
        }
        *n_isect = total;
        if (total > 0x7fffffffLL)
            return fail(XPR_ERR_CAPACITY, "xpr_forward_items: %lld intersections exceed 2^31-1", (long long)total);
        if (total > capacity)
            return fail(XPR_ERR_CAPACITY, "xpr_forward_items: %lld intersections > capacity %lld", (long long)total,
                        (long long)capacity);
        // pairs in depth order with global tile ids, then a stable sort by tile (the key path)
        if (total > 0 &&
            (s = launch_bin_emit_items(rec, bbox, tc, order, cams, items, n_items, *cfg, offsets, tiles, vals_in, st)))
            return s;
        if ((s = launch_sort_tiles(tiles, vals_in, total, (int32_t)S, nullptr, vals, ranges, bin + L.k_sort,
                                   sort_tiles_workspace_bytes(std::max<int64_t>(capacity, 1), (int32_t)S), st)))
            return s;
    }
    if (n_items == 1)  // one item: one block per tile (nothing to balance across items)
        return launch_render_fwd_items(rec, R, vals, ranges, t, *cfg, image, t_final, n_contrib, nullptr, nullptr,
                                       st);
    if ((s = launch_tile_worklist(ranges, (int32_t)S, wl, w + L.wl_ws, worklist_workspace_bytes((int32_t)S), st)))
        return s;
    return launch_render_fwd_items(rec, R, vals, ranges, t, *cfg, image, t_final, n_contrib, wl, counter, st);
}

int xpr_project_color(const float *mu, const float *sh, int64_t n, const XprCamera *cams, int32_t n_views,
                      const XprConfig *cfg, float *rec, void *stream) {
    int s = check_views(n_views, n);
    if (s) return s;
    if (!cams) return fail(XPR_ERR_INVALID, "xpr_project_color: NULL cameras");
    for (int v = 0; v < n_views; ++v)
        if ((s = validate_camera_config(cams + v, cfg))) return s;
    if ((s = need_method(cfg, XPR_METHOD_3DGS, "xpr_project_color"))) return s;
    if (n == 0) return XPR_OK;
    if (!mu || !sh || !rec) return fail(XPR_ERR_INVALID, "xpr_project_color: NULL pointer");
    return launch_project_color_views(mu, sh, n, cams, n_views, *cfg, rec, as_stream(stream));
}

size_t xpr_bin_sorted_workspace(int64_t n, int32_t n_views, const XprCamera *cam, const XprConfig *cfg) {
    if (!cam || !cfg || n < 0 || n_views < 1 || n_views > kMaxViews || validate_camera_config(cam, cfg) != XPR_OK)
        return 0;
    return binsort_workspace_bytes(n, n_views, *cam, *cfg);
}

int xpr_bin_sorted(const float *rec, const int32_t *bbox, const int32_t *tile_count, const int32_t *order, int64_t n,
                   int32_t n_views, const XprCamera *cam, const XprConfig *cfg, int32_t *ranges, uint32_t *vals,
                   int64_t capacity, int64_t *n_isect, void *workspace, size_t ws_bytes, void *stream) {
    int s = validate_camera_config(cam, cfg);
    if (s) return s;
    if ((s = check_views(n_views, n))) return s;
    if (cfg->method == XPR_METHOD_LINPRIM)
        return fail(XPR_ERR_INVALID, "xpr_bin_sorted: LinPrim is binned by xpr_tile_bin_lp");
    if (!binsort_supported(*cam, *cfg, n_views))
        return fail(XPR_ERR_INVALID, "xpr_bin_sorted: a %d x %d tile grid (x %d views) has more than 4096 tile columns",
                    tiles_x(*cam, *cfg), tiles_y(*cam, *cfg), n_views);
    if (!ranges || !n_isect) return fail(XPR_ERR_INVALID, "xpr_bin_sorted: NULL ranges or n_isect");
    if (capacity < 0) return fail(XPR_ERR_INVALID, "xpr_bin_sorted: negative capacity");
    if (n > 0 && (!rec || !bbox || !tile_count || !order || !workspace))
        return fail(XPR_ERR_INVALID, "xpr_bin_sorted: NULL pointer");
    if (n > 0 && (!aligned(rec, 16) || !aligned(bbox, 16) || !aligned(workspace, 256)))
        return fail(XPR_ERR_INVALID, "xpr_bin_sorted: rec/bbox must be 16-byte and workspace 256-byte aligned");
    return launch_binsort(rec, bbox, tile_count, order, n, n_views, *cam, *cfg, ranges, vals, capacity, n_isect,
                          workspace, ws_bytes, as_stream(stream));
}

size_t xpr_bin_rows_workspace(int64_t n, int64_t n_spans, int64_t n_isect, const XprCamera *cam,
                              const XprConfig *cfg) {
    return xpr_bin_rows_views_workspace(n, 1, n_spans, n_isect, cam, cfg);
}

// Shared argument checks and launch of the three rows binning entries (n_rec records, table t).
static int bin_rows_call(const char *fn, const float *rec, const int32_t *bbox, const int32_t *tile_count,
                         const int32_t *isect_count, const int32_t *order, int64_t n_rec, const RowItems &t,
                         const XprConfig *cfg, int32_t *ranges, uint32_t *vals, int64_t capacity, int64_t *n_isect,
                         int64_t *n_spans, void *workspace, size_t ws_bytes, void *stream) {
    if (cfg->method == XPR_METHOD_LINPRIM) return fail(XPR_ERR_INVALID, "%s: LinPrim is binned by xpr_tile_bin_lp", fn);
    if (!bin_rows_supported(t))
        return fail(XPR_ERR_INVALID, "%s: a tile grid has more than 128 tile columns or rows", fn);
    if (!ranges || !n_isect || !n_spans) return fail(XPR_ERR_INVALID, "%s: NULL ranges, n_isect or n_spans", fn);
    if (capacity < 0) return fail(XPR_ERR_INVALID, "%s: negative capacity", fn);
    if (n_rec > 0 && (!rec || !bbox || !tile_count || !order || !workspace || (capacity > 0 && !vals)))
        return fail(XPR_ERR_INVALID, "%s: NULL pointer", fn);
    if (n_rec > 0 && (!aligned(rec, 16) || !aligned(bbox, 16) || !aligned(workspace, 256)))
        return fail(XPR_ERR_INVALID, "%s: rec/bbox must be 16-byte and workspace 256-byte aligned", fn);
    return launch_bin_rows(rec, bbox, tile_count, isect_count, order, n_rec, t, *cfg, ranges, vals, capacity, n_isect,
                           n_spans, workspace, ws_bytes, as_stream(stream));
}

int xpr_bin_rows(const float *rec, const int32_t *bbox, const int32_t *tile_count, const int32_t *isect_count,
                 const int32_t *order, int64_t n, const XprCamera *cam, const XprConfig *cfg, int32_t *ranges,
                 uint32_t *vals, int64_t capacity, int64_t *n_isect, int64_t *n_spans, void *workspace,
                 size_t ws_bytes, void *stream) {
    int s = validate_camera_config(cam, cfg);
    if (s) return s;
    if ((s = check_n(n))) return s;
    return bin_rows_call("xpr_bin_rows", rec, bbox, tile_count, isect_count, order, n,
                         row_items_views(*cam, *cfg, n, 1), cfg, ranges, vals, capacity, n_isect, n_spans, workspace,
                         ws_bytes, stream);
}

size_t xpr_bin_rows_views_workspace(int64_t n, int32_t n_views, int64_t n_spans, int64_t n_isect,
                                    const XprCamera *cam, const XprConfig *cfg) {
    if (validate_camera_config(cam, cfg) != XPR_OK || n < 0 || n_views < 1 || n_views > kMaxViews ||
        n * (int64_t)n_views > 0x7fffffffLL || n_spans < 0 || n_isect < 0)
        return 0;
    const RowItems t = row_items_views(*cam, *cfg, n, n_views);
    if (!bin_rows_supported(t)) return 0;
    return bin_rows_workspace_bytes(n * n_views, n_spans, n_isect, t);
}

int xpr_bin_rows_views(const float *rec, const int32_t *bbox, const int32_t *tile_count, const int32_t *isect_count,
                       const int32_t *order, int64_t n, int32_t n_views, const XprCamera *cam, const XprConfig *cfg,
                       int32_t *ranges, uint32_t *vals, int64_t capacity, int64_t *n_isect, int64_t *n_spans,
                       void *workspace, size_t ws_bytes, void *stream) {
    int s = validate_camera_config(cam, cfg);
    if (s) return s;
    if ((s = check_views(n_views, n))) return s;
    return bin_rows_call("xpr_bin_rows_views", rec, bbox, tile_count, isect_count, order, n * n_views,
                         row_items_views(*cam, *cfg, n, n_views), cfg, ranges, vals, capacity, n_isect, n_spans,
                         workspace, ws_bytes, stream);
}

size_t xpr_bin_rows_items_workspace(const XprCamera *cams, const XprItem *items, int32_t n_items,
                                    const XprConfig *cfg, int64_t n_spans, int64_t n_isect) {
    ItemTable it;
    int64_t R = 0;
    if (!cfg || n_spans < 0 || n_isect < 0 ||
        make_item_table(cams, items, n_items, *cfg, it, &R, "xpr_bin_rows_items_workspace") != XPR_OK)
        return 0;
    const RowItems t = row_items_items(cams, items, n_items, *cfg);
    if (!bin_rows_supported(t)) return 0;
    return bin_rows_workspace_bytes(R, n_spans, n_isect, t);
}

int xpr_bin_rows_items(const float *rec, const int32_t *bbox, const int32_t *tile_count, const int32_t *isect_count,
                       const int32_t *order, const XprCamera *cams, const XprItem *items, int32_t n_items,
                       const XprConfig *cfg, int32_t *ranges, uint32_t *vals, int64_t capacity, int64_t *n_isect,
                       int64_t *n_spans, void *workspace, size_t ws_bytes, void *stream) {
    if (!cfg) return fail(XPR_ERR_INVALID, "xpr_bin_rows_items: NULL config");
    ItemTable it;
    int64_t R = 0;
    int s = make_item_table(cams, items, n_items, *cfg, it, &R, "xpr_bin_rows_items");
    if (s) return s;
    return bin_rows_call("xpr_bin_rows_items", rec, bbox, tile_count, isect_count, order, R,
                         row_items_items(cams, items, n_items, *cfg), cfg, ranges, vals, capacity, n_isect, n_spans,
                         workspace, ws_bytes, stream);
}

// ---- 3DGUT --------------------------------------------------------------------------------

int xpr_project_ut(const XprPrims *prims, int64_t n, const XprCamera *cam, const XprConfig *cfg, float *rec,
                   float *sd, int32_t *bbox, int32_t *tile_count, int32_t *isect_count, void *stream) {
    int s = validate_camera_config(cam, cfg);
    if (s) return s;
    if ((s = need_method(cfg, XPR_METHOD_3DGUT, "xpr_project_ut"))) return s;
    if ((s = check_n(n))) return s;
    if (n == 0) return XPR_OK;
    if (!prims || !prims->mu || !prims->scale || !prims->quat || !prims->opacity || !prims->sh || !rec || !sd ||
        !bbox || !tile_count)
        return fail(XPR_ERR_INVALID, "xpr_project_ut: NULL pointer");
    if (!aligned(prims->quat, 16) || !aligned(rec, 16) || !aligned(sd, 16) || !aligned(bbox, 16))
        return fail(XPR_ERR_INVALID, "xpr_project_ut: quat, rec, sd and bbox must be 16-byte aligned");
    return launch_ut_project_fwd_views(*prims, n, cam, 1, *cfg, rec, sd, bbox, tile_count, isect_count,
                                       as_stream(stream));
}

int xpr_render_ut_fwd(const float *sd, int64_t n, const uint32_t *vals, const int32_t *ranges, const XprCamera *cam,
                      const XprConfig *cfg, float *image, float *t_final, int32_t *n_contrib, void *stream) {
    int s = validate_camera_config(cam, cfg);
    if (s) return s;
    if ((s = need_method(cfg, XPR_METHOD_3DGUT, "xpr_render_ut_fwd"))) return s;
    if ((s = check_n(n))) return s;
    if (!ranges || !image || !t_final || !n_contrib) return fail(XPR_ERR_INVALID, "xpr_render_ut_fwd: NULL pointer");
    if (n > 0 && (!sd || !aligned(sd, 16))) return fail(XPR_ERR_INVALID, "xpr_render_ut_fwd: sd NULL or unaligned");
    if (!aligned(ranges, 8)) return fail(XPR_ERR_INVALID, "xpr_render_ut_fwd: ranges must be 8-byte aligned");
    return launch_ut_render_fwd(sd, n, vals, ranges, 1, *cam, *cfg, image, t_final, n_contrib, nullptr, nullptr,
                                as_stream(stream));
}

int xpr_render_ut_bwd(const float *sd, int64_t n, const uint32_t *vals, const int32_t *ranges, const XprCamera *cam,
                      const XprConfig *cfg, const float *t_final, const int32_t *n_contrib, const float *d_image,
                      float *d_sd, void *stream) {
    int s = validate_camera_config(cam, cfg);
    if (s) return s;
    if ((s = need_method(cfg, XPR_METHOD_3DGUT, "xpr_render_ut_bwd"))) return s;
    if ((s = check_n(n))) return s;
    if (!ranges || !t_final || !n_contrib || !d_image) return fail(XPR_ERR_INVALID, "xpr_render_ut_bwd: NULL pointer");
    if (n == 0) return XPR_OK;
    if (!sd || !d_sd || !aligned(sd, 16) || !aligned(d_sd, 16))
        return fail(XPR_ERR_INVALID, "xpr_render_ut_bwd: sd/d_sd NULL or not 16-byte aligned");
    if (!aligned(ranges, 8)) return fail(XPR_ERR_INVALID, "xpr_render_ut_bwd: ranges must be 8-byte aligned");
    return launch_ut_render_bwd(sd, n, vals, ranges, 1, *cam, *cfg, t_final, n_contrib, d_image, d_sd, nullptr,
                                nullptr, as_stream(stream));
}

int xpr_project_ut_bwd(const XprPrims *prims, int64_t n, const XprCamera *cam, const XprConfig *cfg,
                       const float *d_sd, const XprPrimsGrad *d_prims, void *stream) {
    int s = validate_camera_config(cam, cfg);
    if (s) return s;
    if ((s = need_method(cfg, XPR_METHOD_3DGUT, "xpr_project_ut_bwd"))) return s;
    if ((s = check_n(n))) return s;
    if (n == 0) return XPR_OK;
    if (!prims || !d_prims || !d_sd || !prims->mu || !prims->scale || !prims->quat || !prims->opacity ||
        !prims->sh || !d_prims->mu || !d_prims->scale || !d_prims->quat || !d_prims->opacity || !d_prims->sh)
        return fail(XPR_ERR_INVALID, "xpr_project_ut_bwd: NULL pointer");
    if (!aligned(prims->quat, 16) || !aligned(d_prims->quat, 16) || !aligned(d_sd, 16))
        return fail(XPR_ERR_INVALID, "xpr_project_ut_bwd: quat and d_sd must be 16-byte aligned");
    return launch_ut_project_bwd_views(*prims, n, cam, 1, *cfg, d_sd, *d_prims, as_stream(stream));
}

// ---- 3DGUT, multi-view form ---------------------------------------------------------------

int xpr_project_ut_views(const XprPrims *prims, int64_t n, const XprCamera *cams, int32_t n_views,
                         const XprConfig *cfg, float *rec, float *sd, int32_t *bbox, int32_t *tile_count,
                         int32_t *isect_count, void *stream) {
    int s = check_views(n_views, n);
    if (s) return s;
    if (!cams) return fail(XPR_ERR_INVALID, "xpr_project_ut_views: NULL cameras");
    for (int v = 0; v < n_views; ++v)
        if ((s = validate_camera_config(cams + v, cfg))) return s;
    if ((s = need_method(cfg, XPR_METHOD_3DGUT, "xpr_project_ut_views"))) return s;
    if (n == 0) return XPR_OK;
    if (!prims || !prims->mu || !prims->scale || !prims->quat || !prims->opacity || !prims->sh || !rec || !sd ||
        !bbox || !tile_count)
        return fail(XPR_ERR_INVALID, "xpr_project_ut_views: NULL pointer");
    if (!aligned(prims->quat, 16) || !aligned(rec, 16) || !aligned(sd, 16) || !aligned(bbox, 16))
        return fail(XPR_ERR_INVALID, "xpr_project_ut_views: quat, rec, sd and bbox must be 16-byte aligned");
    return launch_ut_project_fwd_views(*prims, n, cams, n_views, *cfg, rec, sd, bbox, tile_count, isect_count,
                                       as_stream(stream));
}

int xpr_render_ut_fwd_views(const float *sd, int64_t n, int32_t n_views, const uint32_t *vals, const int32_t *ranges,
                            const XprCamera *cam, const XprConfig *cfg, float *image, float *t_final,
                            int32_t *n_contrib, const int32_t *worklist, int32_t *counter, void *stream) {
    int s = validate_camera_config(cam, cfg);
    if (s) return s;
    if ((s = need_method(cfg, XPR_METHOD_3DGUT, "xpr_render_ut_fwd_views"))) return s;
    if ((s = check_views(n_views, n))) return s;
    if (!ranges || !image || !t_final || !n_contrib) return fail(XPR_ERR_INVALID, "xpr_render_ut_fwd_views: NULL");
    if (n > 0 && (!sd || !aligned(sd, 16))) return fail(XPR_ERR_INVALID, "xpr_render_ut_fwd_views: sd");
    if (worklist && !counter) return fail(XPR_ERR_INVALID, "xpr_render_ut_fwd_views: worklist needs a counter");
    if (!aligned(ranges, 8)) return fail(XPR_ERR_INVALID, "xpr_render_ut_fwd_views: ranges must be 8-byte aligned");
    return launch_ut_render_fwd(sd, n * n_views, vals, ranges, n_views, *cam, *cfg, image, t_final, n_contrib,
                                worklist, counter, as_stream(stream));
}

int xpr_render_ut_bwd_views(const float *sd, int64_t n, int32_t n_views, const uint32_t *vals, const int32_t *ranges,
                            const XprCamera *cam, const XprConfig *cfg, const float *t_final,
                            const int32_t *n_contrib, const float *d_image, float *d_sd, const int32_t *worklist,
                            int32_t *counter, void *stream) {
    int s = validate_camera_config(cam, cfg);
    if (s) return s;
    if ((s = need_method(cfg, XPR_METHOD_3DGUT, "xpr_render_ut_bwd_views"))) return s;
    if ((s = check_views(n_views, n))) return s;
    if (!ranges || !t_final || !n_contrib || !d_image) return fail(XPR_ERR_INVALID, "xpr_render_ut_bwd_views: NULL");
    if (n == 0) return XPR_OK;
    if (!sd || !d_sd || !aligned(sd, 16) || !aligned(d_sd, 16))
        return fail(XPR_ERR_INVALID, "xpr_render_ut_bwd_views: sd/d_sd NULL or not 16-byte aligned");
    if (worklist && !counter) return fail(XPR_ERR_INVALID, "xpr_render_ut_bwd_views: worklist needs a counter");
    if (!aligned(ranges, 8)) return fail(XPR_ERR_INVALID, "xpr_render_ut_bwd_views: ranges must be 8-byte aligned");
    return launch_ut_render_bwd(sd, n * n_views, vals, ranges, n_views, *cam, *cfg, t_final, n_contrib, d_image,
                                d_sd, worklist, counter, as_stream(stream));
}

int xpr_project_ut_bwd_views(const XprPrims *prims, int64_t n, const XprCamera *cams, int32_t n_views,
                             const XprConfig *cfg, const float *d_sd, const XprPrimsGrad *d_prims, void *stream) {
    int s = check_views(n_views, n);
    if (s) return s;
    if (!cams) return fail(XPR_ERR_INVALID, "xpr_project_ut_bwd_views: NULL cameras");
    for (int v = 0; v < n_views; ++v)
        if ((s = validate_camera_config(cams + v, cfg))) return s;
    if ((s = need_method(cfg, XPR_METHOD_3DGUT, "xpr_project_ut_bwd_views"))) return s;
    if (n == 0) return XPR_OK;
    if (!prims || !d_prims || !d_sd || !prims->mu || !prims->scale || !prims->quat || !prims->opacity ||
        !prims->sh || !d_prims->mu || !d_prims->scale || !d_prims->quat || !d_prims->opacity || !d_prims->sh)
        return fail(XPR_ERR_INVALID, "xpr_project_ut_bwd_views: NULL pointer");
    if (!aligned(prims->quat, 16) || !aligned(d_prims->quat, 16) || !aligned(d_sd, 16))
        return fail(XPR_ERR_INVALID, "xpr_project_ut_bwd_views: quat and d_sd must be 16-byte aligned");
    return launch_ut_project_bwd_views(*prims, n, cams, n_views, *cfg, d_sd, *d_prims, as_stream(stream));
}

// ---- LinPrim ------------------------------------------------------------------------------

int xpr_project_lp(const XprPrims *prims, int64_t n, const XprCamera *cam, const XprConfig *cfg, float *rec,
                   float *sd, int32_t *bbox, int32_t *tile_count, int32_t *isect_count, void *stream) {
    int s = validate_camera_config(cam, cfg);
    if (s) return s;
    if ((s = need_method(cfg, XPR_METHOD_LINPRIM, "xpr_project_lp"))) return s;
    if ((s = check_n(n))) return s;
    if (n == 0) return XPR_OK;
    if (!prims || !prims->mu || !prims->scale || !prims->quat || !prims->opacity || !prims->sh || !rec || !sd ||
        !bbox || !tile_count)
        return fail(XPR_ERR_INVALID, "xpr_project_lp: NULL pointer");
    if (!aligned(prims->quat, 16) || !aligned(rec, 16) || !aligned(sd, 16) || !aligned(bbox, 16))
        return fail(XPR_ERR_INVALID, "xpr_project_lp: quat, rec, sd and bbox must be 16-byte aligned");
    return launch_lp_project_fwd_views(*prims, n, cam, 1, *cfg, rec, sd, bbox, tile_count, isect_count,
                                       as_stream(stream));
}

int xpr_tile_bin_lp(const float *rec, const float *sd, const int32_t *bbox, const int32_t *tile_count,
                    const int32_t *isect_count, const int32_t *order, int64_t n, const XprCamera *cam,
                    const XprConfig *cfg, int32_t *offsets, uint64_t *keys, uint32_t *tiles, uint32_t *vals,
                    int64_t capacity, int64_t *n_isect, void *workspace, size_t ws_bytes, void *stream) {
    if (n > 0 && !sd) return fail(XPR_ERR_INVALID, "xpr_tile_bin_lp: NULL sd");
    static const float kNoData = 0.f;  // stands in for sd when n == 0
    return tile_bin_impl(rec, bbox, tile_count, isect_count, order, n, cam, cfg, offsets, keys, tiles, vals,
                         capacity, n_isect, workspace, ws_bytes, stream, 0, n > 0 ? sd : &kNoData);
}

int xpr_render_lp_fwd(const float *sd, int64_t n, const uint32_t *vals, const int32_t *ranges, const XprCamera *cam,
                      const XprConfig *cfg, float *image, float *t_final, int32_t *n_contrib, void *stream) {
    int s = validate_camera_config(cam, cfg);
    if (s) return s;
    if ((s = need_method(cfg, XPR_METHOD_LINPRIM, "xpr_render_lp_fwd"))) return s;
    if ((s = check_n(n))) return s;
    if (!ranges || !image || !t_final || !n_contrib) return fail(XPR_ERR_INVALID, "xpr_render_lp_fwd: NULL pointer");
    if (n > 0 && (!sd || !aligned(sd, 16))) return fail(XPR_ERR_INVALID, "xpr_render_lp_fwd: sd NULL or unaligned");
    if (!aligned(ranges, 8)) return fail(XPR_ERR_INVALID, "xpr_render_lp_fwd: ranges must be 8-byte aligned");
    return launch_lp_render_fwd(sd, n, vals, ranges, 1, *cam, *cfg, image, t_final, n_contrib, nullptr, nullptr,
                                as_stream(stream));
}

int xpr_render_lp_bwd(const float *sd, int64_t n, const uint32_t *vals, const int32_t *ranges, const XprCamera *cam,
                      const XprConfig *cfg, const float *t_final, const int32_t *n_contrib, const float *d_image,
                      float *d_sd, void *stream) {
    int s = validate_camera_config(cam, cfg);
    if (s) return s;
    if ((s = need_method(cfg, XPR_METHOD_LINPRIM, "xpr_render_lp_bwd"))) return s;
    if ((s = check_n(n))) return s;
    if (!ranges || !t_final || !n_contrib || !d_image) return fail(XPR_ERR_INVALID, "xpr_render_lp_bwd: NULL pointer");
    if (n == 0) return XPR_OK;
    if (!sd || !d_sd || !aligned(sd, 16) || !aligned(d_sd, 16))
        return fail(XPR_ERR_INVALID, "xpr_render_lp_bwd: sd/d_sd NULL or not 16-byte aligned");
    if (!aligned(ranges, 8)) return fail(XPR_ERR_INVALID, "xpr_render_lp_bwd: ranges must be 8-byte aligned");
    return launch_lp_render_bwd(sd, n, vals, ranges, 1, *cam, *cfg, t_final, n_contrib, d_image, d_sd, nullptr,
                                nullptr, as_stream(stream));
}

int xpr_project_lp_bwd(const XprPrims *prims, int64_t n, const XprCamera *cam, const XprConfig *cfg,
                       const float *d_sd, const XprPrimsGrad *d_prims, void *stream) {
    int s = validate_camera_config(cam, cfg);
    if (s) return s;
    if ((s = need_method(cfg, XPR_METHOD_LINPRIM, "xpr_project_lp_bwd"))) return s;
    if ((s = check_n(n))) return s;
    if (n == 0) return XPR_OK;
    if (!prims || !d_prims || !d_sd || !prims->mu || !prims->scale || !prims->quat || !prims->opacity ||
        !prims->sh || !d_prims->mu || !d_prims->scale || !d_prims->quat || !d_prims->opacity || !d_prims->sh)
        return fail(XPR_ERR_INVALID, "xpr_project_lp_bwd: NULL pointer");
    if (!aligned(prims->quat, 16) || !aligned(d_prims->quat, 16) || !aligned(d_sd, 16))
        return fail(XPR_ERR_INVALID, "xpr_project_lp_bwd: quat and d_sd must be 16-byte aligned");
    return launch_lp_project_bwd_views(*prims, n, cam, 1, *cfg, d_sd, *d_prims, as_stream(stream));
}

// ---- rendered features ----------------------------------------------------------------------

static int check_feat(const char *fn, int64_t n, const float *feat, int32_t n_feat, int32_t with_depth) {
    const int nf = n_feat + (with_depth ? 1 : 0);
    if (n_feat < 0 || nf < 1 || nf > 16)
        return fail(XPR_ERR_INVALID, "%s: n_feat + with_depth = %d out of range [1, 16]", fn, nf);
    if (n > 0 && n_feat > 0 && !feat) return fail(XPR_ERR_INVALID, "%s: NULL feat", fn);
    return XPR_OK;
}

int xpr_render_fwd_feat(const float *rec, int64_t n, const float *feat, int32_t n_feat, int32_t with_depth,
                        const uint32_t *vals, const int32_t *ranges, const XprCamera *cam, const XprConfig *cfg,
                        float *image, float *features, float *t_final, int32_t *n_contrib, void *stream) {
    int s = validate_camera_config(cam, cfg);
    if (s) return s;
    if ((s = need_method(cfg, XPR_METHOD_3DGS, "xpr_render_fwd_feat"))) return s;
    if ((s = check_n(n))) return s;
    if ((s = check_feat("xpr_render_fwd_feat", n, feat, n_feat, with_depth))) return s;
    if (!ranges || !image || !features || !t_final || !n_contrib)
        return fail(XPR_ERR_INVALID, "xpr_render_fwd_feat: NULL pointer");
    if (n > 0 && (!rec || !aligned(rec, 16))) return fail(XPR_ERR_INVALID, "xpr_render_fwd_feat: rec NULL or unaligned");
    if (!aligned(ranges, 8)) return fail(XPR_ERR_INVALID, "xpr_render_fwd_feat: ranges must be 8-byte aligned");
    return launch_render_feat_fwd(rec, n, feat, n_feat, with_depth, vals, ranges, *cam, *cfg, image, features,
                                  t_final, n_contrib, as_stream(stream));
}

int xpr_render_bwd_feat(const float *rec, int64_t n, const float *feat, int32_t n_feat, int32_t with_depth,
                        const uint32_t *vals, const int32_t *ranges, const XprCamera *cam, const XprConfig *cfg,
                        const float *t_final, const int32_t *n_contrib, const float *d_image,
                        const float *d_features, float *d_rec, float *d_feat, void *stream) {
    int s = validate_camera_config(cam, cfg);
    if (s) return s;
    if ((s = need_method(cfg, XPR_METHOD_3DGS, "xpr_render_bwd_feat"))) return s;
    if ((s = check_n(n))) return s;
    if ((s = check_feat("xpr_render_bwd_feat", n, feat, n_feat, with_depth))) return s;
    if (!ranges || !t_final || !n_contrib || !d_image || !d_features)
        return fail(XPR_ERR_INVALID, "xpr_render_bwd_feat: NULL pointer");
    if (n == 0) return XPR_OK;
    if (!rec || !d_rec || !aligned(rec, 16) || !aligned(d_rec, 16))
        return fail(XPR_ERR_INVALID, "xpr_render_bwd_feat: rec/d_rec NULL or not 16-byte aligned");
    if (n_feat > 0 && !d_feat) return fail(XPR_ERR_INVALID, "xpr_render_bwd_feat: NULL d_feat");
    return launch_render_feat_bwd(rec, n, feat, n_feat, with_depth, vals, ranges, *cam, *cfg, t_final, n_contrib,
                                  d_image, d_features, d_rec, d_feat, as_stream(stream));
}

}  // extern "C"
