// Rasterizer, first half (Sec. 4.2): Replicate, Assign tile ID, Cull.
//
// For the primitive i = order[j] at position j and slot r of its half-open tile bounding box
// (row-major, x = xmin + r mod w, y = ymin + r div w, t = y W' + x) the pair is kept iff the
// StopThePop cull (cull.cuh) passes.  Exact per-position counts (from the projection kernel, or
// from the count pass here) are prefix-summed into offsets, then the emit pass writes every kept
// pair at its offset: culled pairs are never written, so the sort moves only survivors.
#include "cull.cuh"
#include "scan.cuh"

namespace xpr {
namespace {

// Count pass (used when the caller has no per-primitive counts): counts[j] = kept tiles of position j.
__global__ void __launch_bounds__(256) bin_count_kernel(const float *__restrict__ rec, const int4 *__restrict__ bbox,
                                                        const int *__restrict__ tcount,
                                                        const int *__restrict__ order, int64_t n, Grid g,
                                                        int32_t *__restrict__ counts) {
    grid_dep_wait();
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int i = 0, area = 0;
    int4 bb = make_int4(0, 0, 0, 0);
    CullData d = {};
    if (j < n) {
        i = order ? order[j] : (int)j;
        area = box_of(bbox, tcount, i, g, bb);
        if (area > 0) d = load_cull(rec, i);
    }
    const int cnt = count_kept_tiles(d, bb, area, g);
    if (j < n) counts[j] = cnt;
}

__device__ __forceinline__ void put_pair(uint64_t *keys, uint32_t *tiles, uint32_t *vals, int64_t pos, uint32_t t,
                                         uint32_t depth_bits, uint32_t i) {
    if (keys) keys[pos] = ((uint64_t)t << 32) | depth_bits;
    if (tiles) tiles[pos] = t;
    vals[pos] = i;
}

// Emit pass.  Warp w of the grid takes the 32 positions w, w + nw, w + 2 nw, ... (nw warps in
// all), so every warp gets primitives from all depths (in depth order the near-camera boxes, which
// hold most pairs, are neighbours and would pile onto a few warps).  The pairs of position j go to
// [offsets[j], offsets[j+1]) in slot order (the box's rows in order, each row's kept span in
// order).  The tile rows of the warp's 32 boxes are spread over the lanes 32 at a time: each lane
// finds its row's kept span (cull.cuh), a warp scan of the span lengths places the rows (each
// position keeps a running output cursor across steps), the non-empty rows are compacted into the
// warp's shared memory, and the warp writes the step's pairs 32 at a time, a lane finding the row
// of its pair from one OR-reduction of the rows' end offsets, so a row's pairs are written by
// consecutive lanes to consecutive addresses.
// keys (u64 tile << 32 | depth bits) and tiles (u32 tile id) are each written when non-NULL.
// Records of a multi-view launch are view-major (record i belongs to view i div per_view) and the
// tile id of a pair is offset by view * tiles_per_view (per_view = 0: a single view).
// ITEMS: records of a multi-scene launch; record i belongs to the item k whose block
// [rec0[k], rec0[k + 1]) holds it, is binned on item k's tile grid and its tile ids are offset by
// tile0[k] (each lane's grid travels with its rows through the shuffles).
struct BinItems {
    int count;
    int64_t rec0[kMaxItems + 1];
    int64_t tile0[kMaxItems];
    int W[kMaxItems], H[kMaxItems], Wt[kMaxItems], Ht[kMaxItems];
};

template <bool ITEMS>
__global__ void __launch_bounds__(256) bin_emit_kernel(const float *__restrict__ rec, const int4 *__restrict__ bbox,
                                                       const int *__restrict__ tcount,
                                                       const int *__restrict__ order, int64_t n, Grid g,
                                                       int64_t per_view, int tiles_per_view, BinItems bi,
                                                       const int32_t *__restrict__ offsets,
                                                       uint64_t *__restrict__ keys, uint32_t *__restrict__ tiles,
                                                       uint32_t *__restrict__ vals) {
    grid_dep_wait();
    __shared__ int4 s_rows[8][32];  // per warp: the compacted rows of the current step
    __shared__ uint32_t s_dbs[8][32];
    const int lane = threadIdx.x & 31;
    const unsigned lt_mask = (1u << lane) - 1u;
    int4 *s_row = s_rows[threadIdx.x >> 5];
    uint32_t *s_db = s_dbs[threadIdx.x >> 5];
    const int64_t nw = (n + 31) / 32;
    const int64_t w = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (w >= nw) return;
    const int64_t j = w + (int64_t)lane * nw;
    int i = 0, area = 0;
    int4 bb = make_int4(0, 0, 0, 0);
    CullData d = {};
    uint32_t depth_bits = 0, tbase = 0;
    int cursor = 0;  // next output slot of this lane's position
    Grid gl = g;     // this lane's tile grid (its item's, for ITEMS)
    if (j < n) {
        i = order ? order[j] : (int)j;
        cursor = offsets[j];
        int k = 0;
        if (ITEMS) {
            while (k + 1 < bi.count && (int64_t)i >= bi.rec0[k + 1]) ++k;
            gl.W = bi.W[k];
            gl.H = bi.H[k];
            gl.Wt = bi.Wt[k];
            gl.Ht = bi.Ht[k];
        }
        area = box_of(bbox, tcount, i, gl, bb);
        if (area > 0) {
            d = load_cull(rec, i);
            depth_bits = __float_as_uint(rec[(size_t)i * XPR_REC_FLOATS + 9]);
            if (ITEMS)
                tbase = (uint32_t)bi.tile0[k];
            else
                tbase = per_view ? (uint32_t)(i / per_view) * (uint32_t)tiles_per_view : 0u;
        }
    }
    const int h = area > 0 ? bb.w - bb.y : 0;
    const int incl = warp_incl_scan(h);
    const int rows = __shfl_sync(kFullMask, incl, 31);
    const int excl = incl - h;
    for (int f0 = 0; f0 < rows; f0 += 32) {
        const int f = f0 + lane;
        const int p = lane_of(incl, f);
        const CullData e = shfl_cull(d, p);
        const int excl_p = __shfl_sync(kFullMask, excl, p);
        const int ty = __shfl_sync(kFullMask, bb.y, p) + f - excl_p;
        const int x0 = __shfl_sync(kFullMask, bb.x, p), x1 = __shfl_sync(kFullMask, bb.z, p);
        Grid ge = g;
        if (ITEMS) {
            ge.W = __shfl_sync(kFullMask, gl.W, p);
            ge.H = __shfl_sync(kFullMask, gl.H, p);
            ge.Wt = __shfl_sync(kFullMask, gl.Wt, p);
        }
        int ka = 0, kb = -1;
        const int c = f < rows ? row_span_in_box(e, ge, ty, x0, x1, ka, kb) : 0;
        const int ci = warp_incl_scan(c);
        const int cx = ci - c;
        // output slot of this row's first pair: the position's cursor plus its earlier rows here
        const int first = max(excl_p - f0, 0);  // lane of the position's first row in this step
        const int out_row = __shfl_sync(kFullMask, cursor, p) + cx - __shfl_sync(kFullMask, cx, first);
        const int total = __shfl_sync(kFullMask, ci, 31);
        const int i_p = __shfl_sync(kFullMask, i, p);
        const uint32_t tb_p = __shfl_sync(kFullMask, tbase, p);
        const uint32_t db_p = __shfl_sync(kFullMask, depth_bits, p);
        // the step's non-empty rows, compacted in row order: first tile, first output slot,
        // primitive, index of the row's first pair in the step
        const unsigned nonempty = __ballot_sync(kFullMask, c > 0);
        if (c > 0) {
            const int slot = __popc(nonempty & lt_mask);
            s_row[slot] = make_int4((int)(tb_p + (uint32_t)(ty * ge.Wt + ka)), out_row, i_p, cx);
            s_db[slot] = db_p;
        }
        __syncwarp();
        for (int k0 = 0; k0 < total; k0 += 32) {
            // pair k lies in the non-empty row whose index is the number of non-empty rows ending
            // at or before k: those ended before this chunk, plus those whose end (one bit each:
            // non-empty rows end at distinct places) falls below this lane
            const int k = k0 + lane;
            const int e = ci - k0;
            const unsigned ends = __reduce_or_sync(kFullMask, (c > 0 && e > 0 && e <= 32) ? 1u << (e - 1) : 0u);
            const int row = __popc(__ballot_sync(kFullMask, c > 0 && e <= 0)) + __popc(ends & lt_mask);
            if (k < total) {
                const int4 rr = s_row[row];
                const int in_r = k - rr.w;
                put_pair(keys, tiles, vals, (int64_t)rr.y + in_r, (uint32_t)(rr.x + in_r), keys ? s_db[row] : 0u,
                         (uint32_t)rr.z);
            }
        }
        __syncwarp();  // the next step rewrites this warp's rows
        // advance each position's cursor by its rows' pairs in this step
        const int lo = max(excl - f0, 0), hi = min(incl - 1 - f0, 31);
        const int s_hi = __shfl_sync(kFullMask, ci, max(hi, 0));
        const int s_lo = __shfl_sync(kFullMask, ci, max(lo - 1, 0));
        if (h > 0 && hi >= 0 && lo <= 31 && lo <= hi) cursor += s_hi - (lo > 0 ? s_lo : 0);
    }
}

// Sort key of the depth order: camera-z bits of primitives that have tiles, all ones otherwise
// (those go last, in index order).  Depth of a primitive with tiles is > z_near > 0, so its float
// bits order like the values.
// Multi-view: the view of record i (i div per_view) goes in bits 32.. so views stay in order.
__global__ void depth_key_kernel(const float *__restrict__ rec, const int *__restrict__ tcount, int64_t n,
                                 int64_t per_view, uint64_t *__restrict__ keys, uint32_t *__restrict__ vals) {
    grid_dep_wait();
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint64_t view = per_view ? (uint64_t)(i / per_view) : 0ull;
    const uint64_t d = tcount[i] > 0 ? (uint64_t)__float_as_uint(rec[(size_t)i * XPR_REC_FLOATS + 9]) : 0xffffffffull;
    keys[i] = (view << 32) | d;
    vals[i] = (uint32_t)i;
}

// One view: the 32-bit key alone (half the key traffic of the sort's passes).
__global__ void depth_key32_kernel(const float *__restrict__ rec, const int *__restrict__ tcount, int64_t n,
                                   uint32_t *__restrict__ keys, uint32_t *__restrict__ vals) {
    grid_dep_wait();
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    keys[i] = tcount[i] > 0 ? __float_as_uint(rec[(size_t)i * XPR_REC_FLOATS + 9]) : 0xffffffffu;
    vals[i] = (uint32_t)i;
}

// Multi-scene items: the item of record i (its block [rec0[k], rec0[k + 1])) goes in bits 32..
struct KeyItems {
    int count;
    int64_t rec0[kMaxItems + 1];
};

__global__ void depth_key_items_kernel(const float *__restrict__ rec, const int *__restrict__ tcount, KeyItems ki,
                                       uint64_t *__restrict__ keys, uint32_t *__restrict__ vals) {
    grid_dep_wait();
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= ki.rec0[ki.count]) return;
    int k = 0;
    while (k + 1 < ki.count && i >= ki.rec0[k + 1]) ++k;
    const uint64_t d = tcount[i] > 0 ? (uint64_t)__float_as_uint(rec[(size_t)i * XPR_REC_FLOATS + 9]) : 0xffffffffull;
    keys[i] = ((uint64_t)k << 32) | d;
    vals[i] = (uint32_t)i;
}

// ---- device-wide exclusive scan (scan.cuh) ----
// Items of the offsets scans: in[j], or in[gather[j]] gathered through the emission order.
struct ScanArray {
    const int32_t *in;
    __device__ __forceinline__ int32_t operator()(int64_t j) const { return in[j]; }
};
struct ScanGather {
    const int32_t *in;
    const int32_t *gather;
    __device__ __forceinline__ int32_t operator()(int64_t j) const { return in[gather[j]]; }
};

}  // namespace

constexpr int kScanTile = scan_detail::kTile;

int64_t *scan_total_ptr(void *partials, int64_t n) {
    return reinterpret_cast<int64_t *>(partials) + (n + kScanTile - 1) / kScanTile + 1;
}

size_t scan_partials_bytes(int64_t n) {
    int64_t nb = (n + kScanTile - 1) / kScanTile;
    return (size_t)((nb + 2) * sizeof(int64_t) + 255) / 256 * 256;
}

// partials layout: [nb] block sums, then the total (device int64) if total_out is NULL.
int launch_exclusive_scan(const int32_t *in, int32_t *out, int64_t n, void *partials, int64_t *total_out,
                          cudaStream_t st, const int32_t *gather) {
    if (gather) return launch_scan(ScanGather{in, gather}, out, n, partials, total_out, st);
    return launch_scan(ScanArray{in}, out, n, partials, total_out, st);
}

int launch_bin_count(const float *rec, const int32_t *bbox, const int32_t *tc, const int32_t *order, int64_t n,
                     const XprCamera &cam, const XprConfig &cfg, int32_t *counts, cudaStream_t st) {
    if (n == 0) return XPR_OK;
    const int tpb = 256;
    XPR_CUDA_TRY(launch_dependent(bin_count_kernel, dim3((unsigned)((n + tpb - 1) / tpb)), dim3(tpb), 0, st, rec,
                                  reinterpret_cast<const int4 *>(bbox), tc, order, n, make_grid(cam, cfg), counts));
    XPR_LAUNCH_CHECK("bin_count_kernel");
    return XPR_OK;
}

int launch_bin_emit(const float *rec, const int32_t *bbox, const int32_t *tc, const int32_t *order, int64_t n,
                    const XprCamera &cam, const XprConfig &cfg, const int32_t *offsets, uint64_t *keys,
                    uint32_t *tiles, uint32_t *vals, cudaStream_t st, int64_t per_view) {
    if (n == 0) return XPR_OK;
    const int tpb = 256;
    const int64_t warps = (n + 31) / 32;
    BinItems bi;
    memset(&bi, 0, sizeof(bi));
    XPR_CUDA_TRY(launch_dependent(bin_emit_kernel<false>, dim3((unsigned)((warps * 32 + tpb - 1) / tpb)), dim3(tpb), 0,
                                  st, rec, reinterpret_cast<const int4 *>(bbox), tc, order, n, make_grid(cam, cfg),
                                  per_view, tiles_x(cam, cfg) * tiles_y(cam, cfg), bi, offsets, keys, tiles, vals));
    XPR_LAUNCH_CHECK("bin_emit_kernel");
    return XPR_OK;
}

// Multi-scene items: every position of order[R] binned on its record's item grid; tile ids global.
int launch_bin_emit_items(const float *rec, const int32_t *bbox, const int32_t *tc, const int32_t *order,
                          const XprCamera *cams, const XprItem *items, int n_items, const XprConfig &cfg,
                          const int32_t *offsets, uint32_t *tiles, uint32_t *vals, cudaStream_t st) {
    BinItems bi;
    memset(&bi, 0, sizeof(bi));
    bi.count = n_items;
    int64_t tile = 0;
    for (int k = 0; k < n_items; ++k) {
        bi.rec0[k] = items[k].rec_offset;
        bi.tile0[k] = tile;
        bi.W[k] = cams[k].width;
        bi.H[k] = cams[k].height;
        bi.Wt[k] = tiles_x(cams[k], cfg);
        bi.Ht[k] = tiles_y(cams[k], cfg);
        tile += (int64_t)bi.Wt[k] * bi.Ht[k];
    }
    const int64_t R = items[n_items - 1].rec_offset + (items[n_items - 1].n + 31) / 32 * 32;
    bi.rec0[n_items] = R;
    if (R == 0) return XPR_OK;
    const int tpb = 256;
    const int64_t warps = (R + 31) / 32;
    XPR_CUDA_TRY(launch_dependent(bin_emit_kernel<true>, dim3((unsigned)((warps * 32 + tpb - 1) / tpb)), dim3(tpb), 0,
                                  st, rec, reinterpret_cast<const int4 *>(bbox), tc, order, R, make_grid(cams[0], cfg),
                                  0, 0, bi, offsets, nullptr, tiles, vals));
    XPR_LAUNCH_CHECK("bin_emit_kernel<items>");
    return XPR_OK;
}

size_t depth_order_workspace_bytes(int64_t n) {
    const size_t a = ((size_t)n * 8 + 255) / 256 * 256, b = ((size_t)n * 4 + 255) / 256 * 256;
    return 2 * a + b + 256 + sort_workspace_bytes(n, kMaxViews);
}

int launch_depth_order(const float *rec, const int32_t *tc, int64_t n, int32_t *order, void *ws, size_t ws_bytes,
                       cudaStream_t st, int64_t per_view, int n_views) {
    if (n == 0) return XPR_OK;
    if (ws_bytes < depth_order_workspace_bytes(n))
        return fail(XPR_ERR_INVALID, "xpr_depth_order: workspace %zu < %zu bytes", ws_bytes,
                    depth_order_workspace_bytes(n));
    if (n_views < 1 || n_views > kMaxViews) return fail(XPR_ERR_INVALID, "xpr_depth_order: bad view count");
    const size_t a = ((size_t)n * 8 + 255) / 256 * 256, b = ((size_t)n * 4 + 255) / 256 * 256;
    char *p = reinterpret_cast<char *>(ws);
    uint64_t *keys = reinterpret_cast<uint64_t *>(p);
    uint32_t *vals = reinterpret_cast<uint32_t *>(p + 2 * a);
    void *sort_ws = p + 2 * a + b + 256;
    if (n_views == 1) {  // the u64 key buffer holds the u32 keys; the u64 sort's scratch the u32 sort's
        uint32_t *k32 = reinterpret_cast<uint32_t *>(keys);
        XPR_CUDA_TRY(launch_dependent(depth_key32_kernel, dim3((unsigned)((n + 255) / 256)), dim3(256), 0, st, rec, tc,
                                      n, k32, vals));
        XPR_LAUNCH_CHECK("depth_key32_kernel");
        return launch_sort_u32_bits(k32, vals, n, 1, 0, 32, nullptr, reinterpret_cast<uint32_t *>(order), nullptr,
                                    sort_ws, sort_workspace_bytes(n, n_views), st);
    }
    XPR_CUDA_TRY(launch_dependent(depth_key_kernel, dim3((unsigned)((n + 255) / 256)), dim3(256), 0, st, rec, tc, n,
                                  per_view, keys, vals));
    XPR_LAUNCH_CHECK("depth_key_kernel");
    // the sort's "tile" is the view: keys (view << 32 | depth bits) sort over 32 + ceil(log2 views) bits;
    // only the order is wanted (no sorted keys, which lets the sort use `keys` as scratch, and no
    // per-view ranges)
    return launch_sort(keys, vals, n, n_views, 0, nullptr, reinterpret_cast<uint32_t *>(order), nullptr, sort_ws,
                       sort_workspace_bytes(n, n_views), st);
}

int launch_depth_order_items(const float *rec, const int32_t *tc, const XprItem *items, int n_items, int32_t *order,
                             void *ws, size_t ws_bytes, cudaStream_t st) {
    KeyItems ki;
    memset(&ki, 0, sizeof(ki));
    ki.count = n_items;
    for (int k = 0; k < n_items; ++k) ki.rec0[k] = items[k].rec_offset;
    const int64_t R = items[n_items - 1].rec_offset + (items[n_items - 1].n + 31) / 32 * 32;
    ki.rec0[n_items] = R;
    if (R == 0) return XPR_OK;
    if (ws_bytes < depth_order_workspace_bytes(R))
        return fail(XPR_ERR_INVALID, "xpr_depth_order_items: workspace %zu < %zu bytes", ws_bytes,
                    depth_order_workspace_bytes(R));
    const size_t a = ((size_t)R * 8 + 255) / 256 * 256, b = ((size_t)R * 4 + 255) / 256 * 256;
    char *p = reinterpret_cast<char *>(ws);
    uint64_t *keys = reinterpret_cast<uint64_t *>(p);
    uint32_t *vals = reinterpret_cast<uint32_t *>(p + 2 * a);
    void *sort_ws = p + 2 * a + b + 256;
    XPR_CUDA_TRY(launch_dependent(depth_key_items_kernel, dim3((unsigned)((R + 255) / 256)), dim3(256), 0, st, rec, tc,
                                  ki, keys, vals));
    XPR_LAUNCH_CHECK("depth_key_items_kernel");
    return launch_sort(keys, vals, R, n_items, 0, nullptr, reinterpret_cast<uint32_t *>(order), nullptr, sort_ws,
                       sort_workspace_bytes(R, n_items), st);
}

}  // namespace xpr
