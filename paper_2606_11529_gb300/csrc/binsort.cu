// Rasterizer, both halves fused (Sec. 4.2 "Replicate, Assign tile ID, Cull" + "Sort and identify
// bounds"): the per-tile lists are written directly in their sorted order, with no key array and
// no radix pass.
//
// Input: the records in emission (depth) order, order[] from xpr_depth_order.  Wanted: for every
// tile, the kept records in that order, i.e. a stable counting sort of the (record, tile) pairs by
// tile.  The cull of Listing 1 tile_cull keeps, in each tile row, one contiguous span of tile
// columns (cull.cuh, row form), so the work is organised by tile rows:
//
//   * the emission positions of a view are cut into chunks of P positions; a block serves one
//     (view, chunk, group of 8 tile rows), one warp per tile row;
//   * the block scans its chunk's positions 1024 at a time: every warp takes 128 consecutive
//     positions and appends each record whose box meets one of the group's rows to a queue per
//     (warp, row), in position order;
//   * the row's warp then takes the queues of warps 0..7 in turn (that is, position order), 32
//     records at a time: each lane computes its record's kept span [ka, kb] in the row;
//   * count pass: a difference array per row (+1 at ka, -1 at kb + 1) gives, after the chunk, the
//     number of kept pairs of every tile of the row in this chunk: one row of a (chunk x tile)
//     count matrix per view;
//   * the matrix is prefix-summed down each tile's column (over the chunks) and across the tiles:
//     each entry becomes the output position of the chunk's first pair on that tile, and the tile
//     ranges [start, end) follow;
//   * emit pass: the same walk with per-row cursors loaded from the matrix; the 32 records' spans
//     are flattened over the lanes 32 pairs at a time, and a pair's rank among the step's pairs on
//     the same tile is the number of lower lanes with the same tile (__match_any_sync): lanes hold
//     the pairs in record order and a record has at most one pair per tile, so those are exactly
//     the earlier records' pairs.  vals[cursor + rank] = record, and the last of them advances the
//     cursor.
// Within a tile, chunks come in position order and a chunk's pairs in record order, so the lists
// are the (tile, depth, index) order of the key sort, bit for bit, with the same kept set.
#include <algorithm>

#include "cull.cuh"

namespace xpr {
namespace {

constexpr int kRows = 8;                 // tile rows per block: one warp each
constexpr int kRound = 1024;             // positions scanned per round (128 per warp)
constexpr int kPerWarp = kRound / kRows;
constexpr int kSegChunks = 32;           // chunks per segment of the column prefix
constexpr int64_t kMinChunk = kRound;  // positions per chunk, at least
constexpr int kColThreads = 256;
constexpr int kMaxCols = 4096;           // tile columns (a 32768-pixel row in 8-pixel tiles)
constexpr int64_t kMatrixEntries = int64_t(16) << 20;  // count-matrix budget (64 MB)

// One item of the walk: a view of the single- / multi-view calls, or a (scene, camera) item of
// the multi-scene call.  Its positions are order[pos0, pos0 + n), its tiles the global ids
// [tile0, tile0 + T), its count matrix mat[mat0 ..] of nc rows by T, its segment sums
// part[part0 ..] of nseg rows by T, and its blocks of the walk grid [blk0, blk0 + nc ng).
struct BItem {
    Grid g;
    int T, nc, ng, nseg, blk0;
    int64_t n, pos0, tile0, mat0, part0;
};

struct Shape {
    int K;          // items
    int64_t P;      // positions per chunk (a multiple of kRound)
    int blocks;     // walk blocks over all items
    int max_T, max_nseg;
    int64_t S;      // tiles over all items
    int64_t mat_entries, part_entries;
    BItem it[kMaxItems];
};

// grids[k], n[k], pos0[k], tile0[k] for k < K; tile0 must be the running sum of the grids' tiles.
Shape make_shape(int K, const Grid *grids, const int64_t *n, const int64_t *pos0) {
    Shape s = {};
    s.K = K;
    // the smallest chunk of at least kMinChunk positions whose count matrix fits the budget (longer
    // per-(chunk, tile) segments keep the scattered writes of the emit pass to fewer partial sectors)
    int64_t P = kMinChunk;
    for (;;) {
        int64_t e = 0;
        for (int k = 0; k < K; ++k)
            e += std::max<int64_t>(1, (n[k] + P - 1) / P) * (int64_t)grids[k].Wt * grids[k].Ht;
        if (e <= kMatrixEntries || P >= (int64_t(1) << 40)) break;
        P += kRound;
    }
    s.P = P;
    int64_t tile0 = 0, mat0 = 0, part0 = 0;
    int blk0 = 0;
    for (int k = 0; k < K; ++k) {
        BItem &b = s.it[k];
        b.g = grids[k];
        b.T = b.g.Wt * b.g.Ht;
        b.n = n[k];
        b.pos0 = pos0[k];
        b.nc = (int)std::max<int64_t>(1, (n[k] + P - 1) / P);
        b.ng = (b.g.Ht + kRows - 1) / kRows;
        b.nseg = (b.nc + kSegChunks - 1) / kSegChunks;
        b.tile0 = tile0;
        b.mat0 = mat0;
        b.part0 = part0;
        b.blk0 = blk0;
        tile0 += b.T;
        mat0 += (int64_t)b.nc * b.T;
        part0 += (int64_t)b.nseg * b.T;
        blk0 += b.nc * b.ng;
        s.max_T = std::max(s.max_T, b.T);
        s.max_nseg = std::max(s.max_nseg, b.nseg);
    }
    s.blocks = blk0;
    s.S = tile0;
    s.mat_entries = mat0;
    s.part_entries = part0;
    return s;
}

Shape make_views_shape(int64_t n, int V, const XprCamera &cam, const XprConfig &cfg) {
    Grid grids[kMaxItems];
    int64_t nn[kMaxItems], p0[kMaxItems];
    for (int v = 0; v < V; ++v) {
        grids[v] = make_grid(cam, cfg);
        nn[v] = n;
        p0[v] = (int64_t)v * n;
    }
    return make_shape(V, grids, nn, p0);
}

struct Ws {
    int32_t *mat;    // count matrix: counts, then first output positions
    int32_t *part;   // segment sums, then segment bases
    int32_t *tot;    // [S + 1]: tile totals, then tile starts
    void *scan;      // scan partials of S entries
};

size_t carve(const Shape &s, void *base, Ws *w) {
    auto up = [](size_t b) { return (b + 255) / 256 * 256; };
    const size_t b_mat = up((size_t)s.mat_entries * sizeof(int32_t));
    const size_t b_part = up((size_t)s.part_entries * sizeof(int32_t));
    const size_t b_tot = up(((size_t)s.S + 1) * sizeof(int32_t));
    const size_t b_scan = up(scan_partials_bytes(s.S));
    if (w) {
        char *p = reinterpret_cast<char *>(base);
        w->mat = reinterpret_cast<int32_t *>(p);
        p += b_mat;
        w->part = reinterpret_cast<int32_t *>(p);
        p += b_part;
        w->tot = reinterpret_cast<int32_t *>(p);
        p += b_tot;
        w->scan = p;
    }
    return b_mat + b_part + b_tot + b_scan;
}

__device__ __forceinline__ int box_rows(const int4 *__restrict__ bbox, const int32_t *__restrict__ tc, int i,
                                        const Grid &g, int4 &bb) {
    bb = make_int4(0, 0, 0, 0);
    if (tc[i] <= 0) return 0;
    bb = bbox[i];
    bb.x = max(bb.x, 0);  // never leave the tile grid, whatever the caller's boxes say
    bb.y = max(bb.y, 0);
    bb.z = min(bb.z, g.Wt);
    bb.w = min(bb.w, g.Ht);
    return (bb.z > bb.x && bb.w > bb.y) ? 1 : 0;
}

// One (item, chunk, row group) per block, kRows warps.  EMIT = false: count pass (writes the
// chunk's row of counts for the group's rows); EMIT = true: writes vals from the cursors in mat.
template <bool EMIT>
__global__ void __launch_bounds__(kRows * 32) rowband_kernel(const float *__restrict__ rec,
                                                             const int4 *__restrict__ bbox,
                                                             const int32_t *__restrict__ tc,
                                                             const int32_t *__restrict__ order, Shape s,
                                                             int32_t *__restrict__ mat, uint32_t *__restrict__ vals,
                                                             int64_t limit) {
    __shared__ int32_t s_q[kRows][kRows][kPerWarp];  // [scanning warp][row] record queue
    __shared__ int32_t s_qn[kRows][kRows];
    extern __shared__ int32_t s_cols[];              // [row][Wt + 1]: difference array / cursors
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const unsigned lt_mask = (1u << lane) - 1u;
    int k = 0;
    while (k + 1 < s.K && (int)blockIdx.x >= s.it[k + 1].blk0) ++k;
    const BItem &it = s.it[k];
    const Grid &g = it.g;
    const int local = (int)blockIdx.x - it.blk0;
    const int c = local / it.ng, g_idx = local - c * it.ng;
    const int row0 = g_idx * kRows;
    const int ty = row0 + wid;
    const bool has_row = ty < g.Ht;
    const int stride = g.Wt + 1;
    int32_t *cols = s_cols + wid * stride;
    int32_t *mrow = mat + it.mat0 + (int64_t)c * it.T + (int64_t)ty * g.Wt;
    for (int x = lane; x < stride; x += 32) cols[x] = (EMIT && has_row && x < g.Wt) ? mrow[x] : 0;
    const int64_t p_begin = (int64_t)c * s.P, p_end = min(p_begin + s.P, it.n);
    const int32_t *ord = order + it.pos0;
    for (int64_t r0 = p_begin; r0 < p_end; r0 += kRound) {
        // scan: warp wid appends the records of positions [r0 + 128 wid, + 128) meeting each row
        int qn[kRows];
#pragma unroll
        for (int r = 0; r < kRows; ++r) qn[r] = 0;
#pragma unroll 1
        for (int itr = 0; itr < kPerWarp / 32; ++itr) {
            const int64_t p = r0 + wid * kPerWarp + itr * 32 + lane;
            int i = 0, has = 0;
            int4 bb = make_int4(0, 0, 0, 0);
            if (p < p_end) {
                i = ord[p];
                has = box_rows(bbox, tc, i, g, bb);
            }
#pragma unroll
            for (int r = 0; r < kRows; ++r) {
                const bool meets = has && row0 + r >= bb.y && row0 + r < bb.w;
                const unsigned m = __ballot_sync(kFullMask, meets);
                if (meets) s_q[wid][r][qn[r] + __popc(m & lt_mask)] = i;
                qn[r] += __popc(m);
            }
        }
        if (lane == 0)
#pragma unroll
            for (int r = 0; r < kRows; ++r) s_qn[wid][r] = qn[r];
        __syncthreads();
        if (has_row) {
            // this row's queue is the scanning warps' sub-queues in order (position order): entry e
            // is sub-queue w's entry e - start[w]
            int qstart[kRows + 1];
            qstart[0] = 0;
#pragma unroll
            for (int w = 0; w < kRows; ++w) qstart[w + 1] = qstart[w] + s_qn[w][wid];
            const int cnt = qstart[kRows];
            for (int e0 = 0; e0 < cnt; e0 += 32) {
                const int e = e0 + lane;
                int i = 0, ka = 0, kb = -1, span = 0;
                if (e < cnt) {
                    int w = 0, off = 0;
#pragma unroll
                    for (int q = 1; q < kRows; ++q)
                        if (e >= qstart[q]) {
                            w = q;
                            off = qstart[q];
                        }
                    i = s_q[w][wid][e - off];
                    const int4 bb = bbox[i];
                    const CullData d = load_cull(rec, i);
                    span = row_span_in_box(d, g, ty, max(bb.x, 0), min(bb.z, g.Wt), ka, kb);
                }
                if (!EMIT) {
                    if (span > 0) {
                        atomicAdd(cols + ka, 1);
                        atomicAdd(cols + kb + 1, -1);
                    }
                    continue;
                }
                const int incl = warp_incl_scan(span);
                const int excl = incl - span;
                const int total = __shfl_sync(kFullMask, incl, 31);
                for (int k0 = 0; k0 < total; k0 += 32) {
                    const int kk = k0 + lane;
                    const int sl = lane_of(incl, min(kk, total - 1));  // lane holding pair kk's record
                    const int tx = __shfl_sync(kFullMask, ka, sl) + (kk - __shfl_sync(kFullMask, excl, sl));
                    const int rid = __shfl_sync(kFullMask, i, sl);
                    const unsigned act = __ballot_sync(kFullMask, kk < total);
                    int base = 0, before = 0;
                    bool last = false;
                    if (kk < total) {
                        const unsigned peers = __match_any_sync(act, tx);
                        before = __popc(peers & lt_mask);
                        last = (peers >> lane) == 1u;  // no higher lane on this tile
                        base = cols[tx];
                    }
                    __syncwarp();
                    if (kk < total) {
                        const int64_t at = (int64_t)base + before;
                        if (at < limit) vals[at] = (uint32_t)rid;  // limit: the pair count (defensive)
                        if (last) cols[tx] = base + before + 1;
                    }
                    __syncwarp();
                }
            }
        }
        __syncthreads();  // the next round rewrites the queues
    }
    if (!EMIT && has_row) {
        // prefix of the difference array: the chunk's pairs on each tile of the row
        __syncwarp();
        int carry = 0;
        for (int x0 = 0; x0 < g.Wt; x0 += 32) {
            const int x = x0 + lane;
            const int dv = x < g.Wt ? cols[x] : 0;
            const int sc = warp_incl_scan(dv) + carry;
            if (x < g.Wt) mrow[x] = sc;
            carry = __shfl_sync(kFullMask, sc, 31);
        }
    }
}

// part[seg][t] of item z = sum of the counts of the segment's chunks on tile t.
__global__ void __launch_bounds__(kColThreads) col_part_kernel(const int32_t *__restrict__ mat, Shape s,
                                                               int32_t *__restrict__ part) {
    const BItem &it = s.it[blockIdx.z];
    const int t = blockIdx.x * kColThreads + threadIdx.x;
    const int seg = blockIdx.y;
    if (t >= it.T || seg >= it.nseg) return;
    const int c0 = seg * kSegChunks, nc = min(kSegChunks, it.nc - c0);
    const int32_t *m = mat + it.mat0 + (int64_t)c0 * it.T + t;
    int sum = 0;
#pragma unroll
    for (int c = 0; c < kSegChunks; ++c) sum += c < nc ? m[(int64_t)c * it.T] : 0;
    part[it.part0 + (int64_t)seg * it.T + t] = sum;
}

// Per tile: exclusive prefix over the segments (in place) and the tile's total.
__global__ void __launch_bounds__(kColThreads) col_seg_kernel(int32_t *__restrict__ part, Shape s,
                                                              int32_t *__restrict__ tot) {
    const BItem &it = s.it[blockIdx.y];
    const int t = blockIdx.x * kColThreads + threadIdx.x;
    if (t >= it.T) return;
    int32_t *p = part + it.part0 + t;
    int run = 0;
    for (int seg = 0; seg < it.nseg; ++seg, p += it.T) {
        const int x = *p;
        *p = run;
        run += x;
    }
    tot[it.tile0 + t] = run;
}

// Counts -> output position of each (chunk, tile)'s first pair; the first segment also writes the
// tile ranges (an empty tile gets [0, 0), as from the key sort's segment search).
__global__ void __launch_bounds__(kColThreads) col_apply_kernel(int32_t *__restrict__ mat,
                                                                const int32_t *__restrict__ part,
                                                                const int32_t *__restrict__ start, Shape s,
                                                                int2 *__restrict__ ranges) {
    const BItem &it = s.it[blockIdx.z];
    const int t = blockIdx.x * kColThreads + threadIdx.x;
    const int seg = blockIdx.y;
    if (t >= it.T || seg >= it.nseg) return;
    const int64_t gt = it.tile0 + t;
    if (seg == 0) {
        const int a = start[gt], b = start[gt + 1];
        ranges[gt] = b > a ? make_int2(a, b) : make_int2(0, 0);
    }
    const int c0 = seg * kSegChunks, nc = min(kSegChunks, it.nc - c0);
    int run = start[gt] + part[it.part0 + (int64_t)seg * it.T + t];
    int32_t *m = mat + it.mat0 + (int64_t)c0 * it.T + t;
    int x[kSegChunks];  // all loads issued before the first store (they do not wait on each other)
#pragma unroll
    for (int c = 0; c < kSegChunks; ++c) x[c] = c < nc ? m[(int64_t)c * it.T] : 0;
#pragma unroll
    for (int c = 0; c < kSegChunks; ++c) {
        if (c < nc) m[(int64_t)c * it.T] = run;
        run += x[c];
    }
}

int run_binsort(const Shape &s, const float *rec, const int32_t *bbox, const int32_t *tc, const int32_t *order,
                int32_t *ranges, uint32_t *vals, int64_t capacity, int64_t *n_isect, void *ws, size_t ws_bytes,
                cudaStream_t st, const char *fn) {
    Ws w;
    const size_t need = carve(s, ws, &w);
    if (ws_bytes < need) return fail(XPR_ERR_INVALID, "%s: workspace %zu < %zu bytes", fn, ws_bytes, need);
    if (s.mat_entries > 0x7fffffffLL || s.S > 0x7fffffffLL || s.blocks < 0)
        return fail(XPR_ERR_INVALID, "%s: too many tiles", fn);
    *n_isect = 0;
    bool any = false;
    int max_wt = 0;
    for (int k = 0; k < s.K; ++k) {
        any |= s.it[k].n > 0;
        max_wt = std::max(max_wt, s.it[k].g.Wt);
    }
    if (!any || s.S == 0) {
        if (s.S) XPR_CUDA_TRY(cudaMemsetAsync(ranges, 0, (size_t)s.S * 2 * sizeof(int32_t), st));
        return XPR_OK;
    }
    // One fixed limit for every call: concurrent callers (other host threads, other grid sizes) must
    // never lower it below what a launch in flight on another stream was checked against.
    const int smem_max = kRows * (kMaxCols + 1) * (int)sizeof(int32_t);
    XPR_CUDA_TRY(cudaFuncSetAttribute(rowband_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_max));
    XPR_CUDA_TRY(cudaFuncSetAttribute(rowband_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_max));
    const size_t smem = (size_t)kRows * (max_wt + 1) * sizeof(int32_t);
    const int4 *bb4 = reinterpret_cast<const int4 *>(bbox);
    rowband_kernel<false><<<(unsigned)s.blocks, kRows * 32, smem, st>>>(rec, bb4, tc, order, s, w.mat, nullptr, 0);
    XPR_LAUNCH_CHECK("rowband_kernel<count>");
    const dim3 cgrid((unsigned)((s.max_T + kColThreads - 1) / kColThreads), (unsigned)s.max_nseg, (unsigned)s.K);
    col_part_kernel<<<cgrid, kColThreads, 0, st>>>(w.mat, s, w.part);
    XPR_LAUNCH_CHECK("col_part_kernel");
    col_seg_kernel<<<dim3(cgrid.x, (unsigned)s.K), kColThreads, 0, st>>>(w.part, s, w.tot);
    XPR_LAUNCH_CHECK("col_seg_kernel");
    int r = launch_exclusive_scan(w.tot, w.tot, s.S, w.scan, nullptr, st);
    if (r) return r;
    col_apply_kernel<<<cgrid, kColThreads, 0, st>>>(w.mat, w.part, w.tot, s, reinterpret_cast<int2 *>(ranges));
    XPR_LAUNCH_CHECK("col_apply_kernel");
    int64_t total = 0;
    XPR_CUDA_TRY(cudaMemcpyAsync(&total, scan_total_ptr(w.scan, s.S), sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    XPR_CUDA_TRY(cudaStreamSynchronize(st));
    *n_isect = total;
    if (total > 0x7fffffffLL)
        return fail(XPR_ERR_CAPACITY, "%s: %lld intersections exceed 2^31-1", fn, (long long)total);
    if (total > capacity)
        return fail(XPR_ERR_CAPACITY, "%s: %lld intersections > capacity %lld", fn, (long long)total,
                    (long long)capacity);
    if (total == 0) return XPR_OK;
    if (!vals) return fail(XPR_ERR_INVALID, "%s: NULL vals", fn);
    rowband_kernel<true><<<(unsigned)s.blocks, kRows * 32, smem, st>>>(rec, bb4, tc, order, s, w.mat, vals, total);
    XPR_LAUNCH_CHECK("rowband_kernel<emit>");
    return XPR_OK;
}

}  // namespace

size_t binsort_workspace_bytes(int64_t n, int n_views, const XprCamera &cam, const XprConfig &cfg) {
    return carve(make_views_shape(n, n_views, cam, cfg), nullptr, nullptr);
}

bool binsort_supported(const XprCamera &cam, const XprConfig &cfg, int n_views) {
    const Grid g = make_grid(cam, cfg);
    return g.Wt <= kMaxCols && n_views >= 1 && n_views <= kMaxViews;
}

int launch_binsort(const float *rec, const int32_t *bbox, const int32_t *tc, const int32_t *order, int64_t n,
                   int n_views, const XprCamera &cam, const XprConfig &cfg, int32_t *ranges, uint32_t *vals,
                   int64_t capacity, int64_t *n_isect, void *ws, size_t ws_bytes, cudaStream_t st) {
    if (n > 0x7fffffffLL) return fail(XPR_ERR_INVALID, "xpr_bin_sorted: %lld records per view", (long long)n);
    return run_binsort(make_views_shape(n, n_views, cam, cfg), rec, bbox, tc, order, ranges, vals, capacity, n_isect,
                       ws, ws_bytes, st, "xpr_bin_sorted");
}

static Shape items_shape(const XprCamera *cams, const XprItem *items, int n_items, const XprConfig &cfg) {
    Grid grids[kMaxItems];
    int64_t nn[kMaxItems], p0[kMaxItems];
    for (int k = 0; k < n_items; ++k) {
        grids[k] = make_grid(cams[k], cfg);
        nn[k] = items[k].n;
        p0[k] = items[k].rec_offset;
    }
    return make_shape(n_items, grids, nn, p0);
}

size_t binsort_items_workspace_bytes(const XprCamera *cams, const XprItem *items, int n_items, const XprConfig &cfg) {
    return carve(items_shape(cams, items, n_items, cfg), nullptr, nullptr);
}

bool binsort_items_supported(const XprCamera *cams, int n_items, const XprConfig &cfg) {
    for (int k = 0; k < n_items; ++k)
        if (make_grid(cams[k], cfg).Wt > kMaxCols) return false;
    return true;
}

int launch_binsort_items(const float *rec, const int32_t *bbox, const int32_t *tc, const int32_t *order,
                         const XprCamera *cams, const XprItem *items, int n_items, const XprConfig &cfg,
                         int32_t *ranges, uint32_t *vals, int64_t capacity, int64_t *n_isect, void *ws,
                         size_t ws_bytes, cudaStream_t st) {
    return run_binsort(items_shape(cams, items, n_items, cfg), rec, bbox, tc, order, ranges, vals, capacity, n_isect,
                       ws, ws_bytes, st, "xpr_bin_sorted_items");
}

}  // namespace xpr
