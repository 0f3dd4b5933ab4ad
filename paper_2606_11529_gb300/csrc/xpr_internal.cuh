// Internal declarations shared by the libxpr translation units (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include "../../include/xpr.h"

namespace xpr {

// ---- error reporting (per host thread) ---------------------------------------------------
void set_error(const char *fmt, ...);
int fail(int status, const char *fmt, ...);
int check_launch(const char *what);

#define XPR_CUDA_TRY(expr)                                                                          \
    do {                                                                                            \
        cudaError_t _e = (expr);                                                                    \
        if (_e != cudaSuccess) return ::xpr::fail(XPR_ERR_CUDA, "%s: %s", #expr, cudaGetErrorString(_e)); \
    } while (0)

#define XPR_LAUNCH_CHECK(what)                  \
    do {                                        \
        int _s = ::xpr::check_launch(what);     \
        if (_s != XPR_OK) return _s;            \
    } while (0)

inline cudaStream_t as_stream(void *s) { return reinterpret_cast<cudaStream_t>(s); }

// Programmatic dependent launch: a kernel launched with launch_dependent may be set up on the
// device while the kernel before it in the stream is still finishing, and waits in grid_dep_wait()
// (its first statement, before any read of what earlier work wrote) until that kernel has
// completed and its writes are visible.  Kernels that call grid_dep_wait() may also be launched
// the ordinary way, where the wait returns at once.
#ifdef __CUDACC__
__device__ __forceinline__ void grid_dep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
#endif
template <typename... Params, typename... Args>
inline cudaError_t launch_dependent(void (*kernel)(Params...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                                    Args... args) {
    cudaLaunchConfig_t c = {};
    c.gridDim = grid;
    c.blockDim = block;
    c.dynamicSmemBytes = smem;
    c.stream = st;
    cudaLaunchAttribute a[1];
    a[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    a[0].val.programmaticStreamSerializationAllowed = 1;
    c.attrs = a;
    c.numAttrs = 1;
    return cudaLaunchKernelEx(&c, kernel, static_cast<Params>(args)...);
}

__host__ __device__ inline int tiles_x(const XprCamera &c, const XprConfig &g) {
    return (c.width + g.tile_w - 1) / g.tile_w;
}
__host__ __device__ inline int tiles_y(const XprCamera &c, const XprConfig &g) {
    return (c.height + g.tile_h - 1) / g.tile_h;
}

int validate_camera_config(const XprCamera *cam, const XprConfig *cfg);

// ---- launch helpers implemented per translation unit -------------------------------------
constexpr int kMaxViews = 16;  // views per multi-view launch (cameras travel as a kernel argument)
constexpr int kMaxItems = 16;  // (scene, camera) items per multi-scene launch

// Per-item tile grids and image placement of a multi-scene launch (count 0: the uniform views of
// one camera size).  Item k owns global tiles [tile0[k], tile0[k + 1]) and the pixels
// [pix0[k], pix0[k] + W[k] H[k]) of the per-pixel buffers (its image planes at 3 pix0[k]).
struct ItemTable {
    int count;
    int W[kMaxItems], H[kMaxItems], Wt[kMaxItems];
    int64_t tile0[kMaxItems + 1];
    int64_t pix0[kMaxItems];
};

// Checks a host item array against its cameras and config (offsets contiguous and in order,
// records aligned to 32) and fills the table; returns an XprStatus.
int make_item_table(const XprCamera *cams, const XprItem *items, int n_items, const XprConfig &cfg,
                    ItemTable &t, int64_t *n_records, const char *fn);
#ifdef __CUDACC__
// The item holding global tile gt (tile0 is increasing; at most kMaxItems items).
__device__ __forceinline__ int item_of_tile(const ItemTable &t, int64_t gt) {
    int k = 0;
#pragma unroll 1
    while (k + 1 < t.count && gt >= t.tile0[k + 1]) ++k;
    return k;
}
#endif

int launch_project_fwd(const XprPrims &p, int64_t n, const XprCamera &cam, const XprConfig &cfg, float *rec,
                       int32_t *bbox, int32_t *tc, int32_t *isect_count, cudaStream_t st,
                       const XprPrimsGrad *copy = nullptr);  // copy: device copy of the geometry read
int launch_project_bwd(const XprPrims &p, int64_t n, const XprCamera &cam, const XprConfig &cfg,
                       const float *d_rec, const XprPrimsGrad &g, cudaStream_t st);
int launch_project_fwd_views(const XprPrims &p, int64_t n, const XprCamera *cams, int n_views, const XprConfig &cfg,
                             float *rec, int32_t *bbox, int32_t *tc, int32_t *isect_count, cudaStream_t st,
                             const XprPrimsGrad *copy = nullptr);
int launch_project_color_views(const float *mu, const float *sh, int64_t n, const XprCamera *cams, int n_views,
                               const XprConfig &cfg, float *rec, cudaStream_t st);
int launch_project_bwd_views(const XprPrims &p, int64_t n, const XprCamera *cams, int n_views, const XprConfig &cfg,
                             const float *d_rec, const XprPrimsGrad &g, cudaStream_t st);
int launch_render_fwd_views(const float *rec, int64_t n, const uint32_t *vals, const int32_t *ranges, int n_views,
                            const XprCamera &cam, const XprConfig &cfg, float *image, float *t_final,
                            int32_t *n_contrib, const int32_t *worklist, int32_t *counter, cudaStream_t st);
int launch_render_bwd_views(const float *rec, const uint32_t *vals, const int32_t *ranges, int n_views,
                            const XprCamera &cam, const XprConfig &cfg, const float *t_final,
                            const int32_t *n_contrib, const float *d_image, float *d_rec, int64_t n,
                            const int32_t *worklist, int32_t *counter, cudaStream_t st);
int launch_project_items(const XprPrims &p, const XprCamera *cams, const XprItem *items, int n_items,
                         const XprConfig &cfg, float *rec, int32_t *bbox, int32_t *tc, cudaStream_t st,
                         int32_t *isect_count = nullptr);
int launch_bin_emit_items(const float *rec, const int32_t *bbox, const int32_t *tc, const int32_t *order,
                          const XprCamera *cams, const XprItem *items, int n_items, const XprConfig &cfg,
                          const int32_t *offsets, uint32_t *tiles, uint32_t *vals, cudaStream_t st);
int launch_project_bwd_items(const XprPrims &p, int64_t n_prims, const XprCamera *cams, const XprItem *items,
                             int n_items, const XprConfig &cfg, const float *d_rec, const XprPrimsGrad &g,
                             cudaStream_t st);
int launch_depth_order_items(const float *rec, const int32_t *tc, const XprItem *items, int n_items, int32_t *order,
                             void *ws, size_t ws_bytes, cudaStream_t st);
int launch_render_fwd_items(const float *rec, int64_t n_rec, const uint32_t *vals, const int32_t *ranges,
                            const ItemTable &it, const XprConfig &cfg, float *image, float *t_final,
                            int32_t *n_contrib, const int32_t *worklist, int32_t *counter, cudaStream_t st);
int launch_render_bwd_items(const float *rec, int64_t n_rec, const uint32_t *vals, const int32_t *ranges,
                            const ItemTable &it, const XprConfig &cfg, const float *t_final,
                            const int32_t *n_contrib, const float *d_image, float *d_rec, const int32_t *worklist,
                            int32_t *counter, cudaStream_t st);
// tiles sorted by descending list length (ranges[t,1] - ranges[t,0]), for persistent scheduling
size_t worklist_workspace_bytes(int32_t n_tiles);
int launch_tile_worklist(const int32_t *ranges, int32_t n_tiles, int32_t *worklist, void *ws, size_t ws_bytes,
                         cudaStream_t st);

// Device-wide exclusive scan of int32 counts: out[j] = sum_{k<j} item(k), out[n] = total, where
// item(k) = in[gather[k]] if gather is non-NULL, else in[k] (then in == out is allowed).
// partials: >= scan_partials_bytes(n) bytes.  total_out: device int64.
size_t scan_partials_bytes(int64_t n);
int64_t *scan_total_ptr(void *partials, int64_t n);  // where the scan leaves the total when total_out == NULL
int launch_exclusive_scan(const int32_t *in, int32_t *out, int64_t n, void *partials, int64_t *total_out,
                          cudaStream_t st, const int32_t *gather = nullptr);

int launch_bin_count(const float *rec, const int32_t *bbox, const int32_t *tc, const int32_t *order, int64_t n,
                     const XprCamera &cam, const XprConfig &cfg, int32_t *counts, cudaStream_t st);
int launch_bin_emit(const float *rec, const int32_t *bbox, const int32_t *tc, const int32_t *order, int64_t n,
                    const XprCamera &cam, const XprConfig &cfg, const int32_t *offsets, uint64_t *keys,
                    uint32_t *tiles, uint32_t *vals, cudaStream_t st, int64_t per_view = 0);
// binning and tile sort by rows (binrows.cu) of one view, of V views of one camera, or of K
// multi-scene items, each grid at most 128 tile columns and rows.  Item k holds the records
// [rec0[k], rec0[k + 1]) and is binned on a W[k] x H[k] image whose tiles are numbered from tile0[k].
struct RowItems {
    int count;
    int64_t rec0[kMaxItems + 1];
    int64_t tile0[kMaxItems + 1];
    int W[kMaxItems], H[kMaxItems], Wt[kMaxItems], Ht[kMaxItems];
};
RowItems row_items_views(const XprCamera &cam, const XprConfig &cfg, int64_t n, int n_views);
RowItems row_items_items(const XprCamera *cams, const XprItem *items, int n_items, const XprConfig &cfg);
bool bin_rows_supported(const XprCamera &cam, const XprConfig &cfg);
bool bin_rows_supported(const RowItems &t);
size_t bin_rows_workspace_bytes(int64_t n_records, int64_t n_spans, int64_t n_isect, const RowItems &t);
int launch_bin_rows(const float *rec, const int32_t *bbox, const int32_t *tc, const int32_t *isect_count,
                    const int32_t *order, int64_t n_records, const RowItems &t, const XprConfig &cfg,
                    int32_t *ranges, uint32_t *vals, int64_t capacity, int64_t *n_isect, int64_t *n_spans, void *ws,
                    size_t ws_bytes, cudaStream_t st);
size_t depth_order_workspace_bytes(int64_t n);
int launch_depth_order(const float *rec, const int32_t *tc, int64_t n, int32_t *order, void *ws, size_t ws_bytes,
                       cudaStream_t st, int64_t per_view = 0, int n_views = 1);

// rendered features (feat.cu)
int launch_render_feat_fwd(const float *rec, int64_t n, const float *feat, int nfeat, int depth, const uint32_t *vals,
                           const int32_t *ranges, const XprCamera &cam, const XprConfig &cfg, float *image,
                           float *features, float *t_final, int32_t *n_contrib, cudaStream_t st);
int launch_render_feat_bwd(const float *rec, int64_t n, const float *feat, int nfeat, int depth, const uint32_t *vals,
                           const int32_t *ranges, const XprCamera &cam, const XprConfig &cfg, const float *t_final,
                           const int32_t *n_contrib, const float *d_image, const float *d_features, float *d_rec,
                           float *d_feat, cudaStream_t st);

// 3DGUT (ut.cu)
int need_method(const XprConfig *cfg, int method, const char *fn);
int launch_ut_project_fwd_views(const XprPrims &p, int64_t n, const XprCamera *cams, int n_views,
                                const XprConfig &cfg, float *rec, float *sd, int32_t *bbox, int32_t *tc,
                                int32_t *isect_count, cudaStream_t st);
int launch_ut_project_bwd_views(const XprPrims &p, int64_t n, const XprCamera *cams, int n_views,
                                const XprConfig &cfg, const float *d_sd, const XprPrimsGrad &g, cudaStream_t st);
int launch_ut_render_fwd(const float *sd, int64_t n, const uint32_t *vals, const int32_t *ranges, int n_views,
                         const XprCamera &cam, const XprConfig &cfg, float *image, float *t_final,
                         int32_t *n_contrib, const int32_t *worklist, int32_t *counter, cudaStream_t st);
int launch_ut_render_bwd(const float *sd, int64_t n, const uint32_t *vals, const int32_t *ranges, int n_views,
                         const XprCamera &cam, const XprConfig &cfg, const float *t_final, const int32_t *n_contrib,
                         const float *d_image, float *d_sd, const int32_t *worklist, int32_t *counter,
                         cudaStream_t st);

// LinPrim (lp.cu)
int launch_lp_project_fwd_views(const XprPrims &p, int64_t n, const XprCamera *cams, int n_views,
                                const XprConfig &cfg, float *rec, float *sd, int32_t *bbox, int32_t *tc,
                                int32_t *isect_count, cudaStream_t st);
int launch_lp_project_bwd_views(const XprPrims &p, int64_t n, const XprCamera *cams, int n_views,
                                const XprConfig &cfg, const float *d_sd, const XprPrimsGrad &g, cudaStream_t st);
int launch_lp_bin_count(const float *sd, const int32_t *bbox, const int32_t *tc, const int32_t *order, int64_t n,
                        const XprCamera &cam, const XprConfig &cfg, int32_t *counts, cudaStream_t st);
int launch_lp_bin_emit(const float *rec, const float *sd, const int32_t *bbox, const int32_t *tc,
                       const int32_t *order, int64_t n, const XprCamera &cam, const XprConfig &cfg,
                       const int32_t *offsets, uint64_t *keys, uint32_t *tiles, uint32_t *vals, cudaStream_t st,
                       int64_t per_view);
int launch_lp_render_fwd(const float *sd, int64_t n, const uint32_t *vals, const int32_t *ranges, int n_views,
                         const XprCamera &cam, const XprConfig &cfg, float *image, float *t_final,
                         int32_t *n_contrib, const int32_t *worklist, int32_t *counter, cudaStream_t st);
int launch_lp_render_bwd(const float *sd, int64_t n, const uint32_t *vals, const int32_t *ranges, int n_views,
                         const XprCamera &cam, const XprConfig &cfg, const float *t_final, const int32_t *n_contrib,
                         const float *d_image, float *d_sd, const int32_t *worklist, int32_t *counter,
                         cudaStream_t st);

// fused bin + sort (binsort.cu)
size_t binsort_workspace_bytes(int64_t n, int n_views, const XprCamera &cam, const XprConfig &cfg);
bool binsort_supported(const XprCamera &cam, const XprConfig &cfg, int n_views);
int launch_binsort(const float *rec, const int32_t *bbox, const int32_t *tc, const int32_t *order, int64_t n,
                   int n_views, const XprCamera &cam, const XprConfig &cfg, int32_t *ranges, uint32_t *vals,
                   int64_t capacity, int64_t *n_isect, void *ws, size_t ws_bytes, cudaStream_t st);

size_t binsort_items_workspace_bytes(const XprCamera *cams, const XprItem *items, int n_items, const XprConfig &cfg);
bool binsort_items_supported(const XprCamera *cams, int n_items, const XprConfig &cfg);
int launch_binsort_items(const float *rec, const int32_t *bbox, const int32_t *tc, const int32_t *order,
                         const XprCamera *cams, const XprItem *items, int n_items, const XprConfig &cfg,
                         int32_t *ranges, uint32_t *vals, int64_t capacity, int64_t *n_isect, void *ws,
                         size_t ws_bytes, cudaStream_t st);

size_t sort_workspace_bytes(int64_t n, int32_t n_tiles);
int launch_sort(const uint64_t *keys_in, const uint32_t *vals_in, int64_t n, int32_t n_tiles, int begin_bit,
                uint64_t *keys_out, uint32_t *vals_out, int32_t *ranges, void *ws, size_t ws_bytes, cudaStream_t st);
size_t sort_tiles_workspace_bytes(int64_t n, int32_t n_tiles);
int sort_device_errors(unsigned *bits);  // synchronises; reads and clears the sort's device flags
int lookback_selftest(uint32_t *zeroed, int max_polls, cudaStream_t st);  // see xpr_selftest_wait
int launch_sort_tiles(const uint32_t *tiles_in, const uint32_t *vals_in, int64_t n, int32_t n_tiles,
                      uint32_t *tiles_out, uint32_t *vals_out, int32_t *ranges, void *ws, size_t ws_bytes,
                      cudaStream_t st);
// stable sort of 4-byte keys by bits [begin_bit, end_bit) (workspace: sort_tiles_workspace_bytes(n, .));
// ranges (NULL: none) are those of the whole key values, 0 .. n_tiles - 1
int launch_sort_u32_bits(const uint32_t *keys_in, const uint32_t *vals_in, int64_t n, int32_t n_tiles, int begin_bit,
                         int end_bit, uint32_t *keys_out, uint32_t *vals_out, int32_t *ranges, void *ws,
                         size_t ws_bytes, cudaStream_t st);

int launch_render_fwd(const float *rec, int64_t n, const uint32_t *vals, const int32_t *ranges,
                      const XprCamera &cam, const XprConfig &cfg, float *image, float *t_final, int32_t *n_contrib,
                      cudaStream_t st);
int launch_render_bwd(const float *rec, const uint32_t *vals, const int32_t *ranges, const XprCamera &cam,
                      const XprConfig &cfg, const float *t_final, const int32_t *n_contrib, const float *d_image,
                      float *d_rec, int64_t n, cudaStream_t st);

// ---- device helpers -----------------------------------------------------------------------
#ifdef __CUDACC__
constexpr float kLog2e = 1.4426950408889634f;  // log2(e)
constexpr float kLn2 = 0.6931471805599453f;    // ln(2)

__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// 1/x to about 1 ulp (the hardware reciprocal; x here is 1 - alpha in [1 - alpha_max, 1]).
__device__ __forceinline__ float rcp_approx(float x) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Staged shading coefficients of one list entry (paper's p_sd with the conic pre-scaled
// by log2(e) so that exp(power) = 2^(A dx^2 + B dx dy + C dy^2)).
struct Shade {
    float mx, my, A, B, C, o, r, g, b;
};

__device__ __forceinline__ Shade load_shade(const float *__restrict__ rec, uint32_t id) {
    const float4 *p = reinterpret_cast<const float4 *>(rec + (size_t)id * XPR_REC_FLOATS);
    float4 a = __ldg(p), b = __ldg(p + 1), c = __ldg(p + 2);
    Shade s;
    s.mx = a.x;
    s.my = a.y;
    s.A = __fmul_rn(-0.5f * kLog2e, a.z);
    s.B = __fmul_rn(-kLog2e, a.w);
    s.C = __fmul_rn(-0.5f * kLog2e, b.x);
    s.o = b.y;
    s.r = b.z;
    s.g = b.w;
    s.b = c.x;
    return s;
}

// Listing 1 evaluate in base-2 form, p = A dx^2 + B dx dy + C dy^2, factored by pixel column: a
// thread's pixels share one column, so A dx^2 and B dx are formed once per (entry, column) and each
// pixel adds (C dy + B dx) dy with two fused multiply-adds.  Every operation is an explicit IEEE
// intrinsic so the forward and the backward kernels compute bit-identical powers and alphas.
struct ColTerms {
    float adx2, bdx;  // A dx^2, B dx
};
__device__ __forceinline__ ColTerms column_terms(float A, float B, float dx) {
    return ColTerms{__fmul_rn(__fmul_rn(A, dx), dx), __fmul_rn(B, dx)};
}
__device__ __forceinline__ float eval_power2(const ColTerms &t, float C, float dy) {
    return __fmaf_rn(__fmaf_rn(C, dy, t.bdx), dy, t.adx2);
}
#endif

}  // namespace xpr
