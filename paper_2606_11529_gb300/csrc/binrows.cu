// Rasterizer first half by rows (Sec. 4.2: Replicate, Assign tile ID, Cull, Sort and identify bounds)
// for one view, for V views of one camera or for K multi-scene items (Sec. 4.3's batches), every
// tile grid at most 128 columns and 128 rows.
//
// The tile cull in row form (cull.cuh) gives, for every primitive and every tile row of its box, one
// interval [ka, kb] of kept tile columns: a span.  The per-tile lists are built from spans:
//   1. span slots: each position j of the depth order owns one slot per row of its box, the slots
//      grouped by row and each row's in depth order.  A count kernel tallies the box rows per
//      (tile row, chunk of 256 depth positions); the exclusive scan of that row-major matrix is
//      where each chunk's slots of each row start;
//   2. the emit kernel writes every slot in place as a 4-byte key (its tile row, or 255 for a row
//      with no kept tile, in bits 0-7; the first kept column in bits 8-14; the number of kept tiles
//      in bits 15-22; the record's item in bits 23-26) and its record as the value: the spans lie
//      as a stable sort of the depth-ordered slots by row would leave them, without the sort;
//   3. an exclusive scan of the span lengths in that order gives every span its first pair: the
//      pairs, were they written out, would be grouped by tile row and, inside a row, by item in
//      depth order (tile code (k << 14) | (tx << 7) | ty); the scan's epilogue marks the first
//      span of every 496-pair sub-window;
//   4. the stable pass by tile column runs on the spans, without expanding them: per window of
//      3968 pairs a histogram of the pairs per column (difference arrays over the spans' column
//      intervals), its column-major scan, and a scatter that ranks each pair among the window's
//      pairs of its column (masks of the spans covering each column, from XOR differences) and
//      writes the records grouped by (column, row, item): every tile (k, tx, ty) one contiguous
//      run, inside it still in depth order, the tile-major depth-sorted list of Sec. 4.2 with no
//      radix pass over the pairs (about seven pairs a span here).
// The tile ranges are found per code where the staged codes change and permuted to the tile ids
// the render uses (item k's tile (tx, ty) at tile0[k] + ty Wt[k] + tx).  The result is identical,
// list for list, to the depth-ordered emission followed by the stable sort of the tile ids.
#include "cull.cuh"
#include "scan.cuh"

namespace xpr {
namespace {

constexpr uint32_t kRowNone = 255;  // key of a span slot whose box row keeps no tile: sorted last
constexpr int kMaxRowGrid = 128;    // tile columns and rows: 7 bits each in the pair's tile code
constexpr int kItemShift = 14;      // the item's bits in the tile code
constexpr int kSpanItemShift = 23;  // and in the span key

// Item of record i (rec0 increasing; at most kMaxItems items).
__device__ __forceinline__ int item_of_record(const RowItems &t, int64_t i) {
    int k = 0;
#pragma unroll 1
    while (k + 1 < t.count && i >= t.rec0[k + 1]) ++k;
    return k;
}

constexpr int kChunk = 256;  // depth positions per chunk of the row grouping (one block, 8 warps)

// This lane's record at depth position j (j < n): its item's grid, clamped tile box and box height.
template <bool ITEMS>
__device__ __forceinline__ int position_box(const int4 *__restrict__ bbox, const int *__restrict__ tcount,
                                            const int *__restrict__ order, int64_t j, const Grid &g,
                                            const RowItems &t, int &i, int &k, Grid &gl, int4 &bb) {
    i = order[j];
    k = 0;
    gl = g;
    if (ITEMS) {
        k = item_of_record(t, i);
        gl.W = t.W[k];
        gl.H = t.H[k];
        gl.Wt = t.Wt[k];
        gl.Ht = t.Ht[k];
    }
    return box_of(bbox, tcount, i, gl, bb) > 0 ? bb.w - bb.y : 0;
}

// count[r * n_chunks + b] = number of box rows at tile row r among the records at depth positions
// [256 b, 256 b + 256): with one slot per box row, the exclusive scan of this row-major matrix is
// where chunk b's slots of row r start when the slots are grouped by row, in depth order.
template <bool ITEMS>
__global__ void __launch_bounds__(kChunk) row_count_kernel(const int4 *__restrict__ bbox,
                                                           const int *__restrict__ tcount,
                                                           const int *__restrict__ order, int64_t n, Grid g,
                                                           RowItems t, int64_t n_chunks, int32_t *__restrict__ count) {
    grid_dep_wait();
    __shared__ int s_cnt[kMaxRowGrid];
    for (int r = threadIdx.x; r < kMaxRowGrid; r += kChunk) s_cnt[r] = 0;
    __syncthreads();
    const int64_t j = (int64_t)blockIdx.x * kChunk + threadIdx.x;
    if (j < n) {
        int i, k;
        Grid gl;
        int4 bb;
        const int h = position_box<ITEMS>(bbox, tcount, order, j, g, t, i, k, gl, bb);
        for (int r = bb.y; r < bb.y + h; ++r) atomicAdd(&s_cnt[r], 1);
    }
    __syncthreads();
    for (int r = threadIdx.x; r < kMaxRowGrid; r += kChunk) count[(int64_t)r * n_chunks + blockIdx.x] = s_cnt[r];
}

struct CountItem {  // the kept tile counts, summed for the pair total
    const int32_t *in;
    __device__ __forceinline__ int32_t operator()(int64_t j) const { return in[j]; }
};

// Block b takes the depth positions [256 b, 256 b + 256), warp w the 32 from 256 b + 32 w, and
// writes each row's span (the row-form cull of one (primitive, tile row)) straight to its place in
// the slots grouped by row: the row's start for this chunk (the scanned count matrix), plus the
// row's slots in the warps before this one, plus those of the lanes before this one in the warp
// (the lane masks per row from XOR differences over the rows).  So every row's spans lie in depth
// order, as a stable sort of depth-ordered slots by row would leave them.  The warp flattens its boxes' rows over its
// lanes; slots at or beyond ns_cap are not written (the launch may precede the check of the slot
// total against the workspace).  With items, each lane's image size and item travel with its rows
// through the shuffles.  pair_total (may be NULL): receives the sum of the kept counts.
template <bool ITEMS>
__global__ void __launch_bounds__(kChunk) span_emit_kernel(const float *__restrict__ rec, const int4 *__restrict__ bbox,
                                                           const int *__restrict__ tcount,
                                                           const int *__restrict__ order, int64_t n, Grid g,
                                                           RowItems t, int64_t n_chunks,
                                                           const int32_t *__restrict__ row0, int64_t ns_cap,
                                                           uint32_t *__restrict__ span_key,
                                                           uint32_t *__restrict__ span_prim,
                                                           unsigned long long *__restrict__ pair_total) {
    grid_dep_wait();
    __shared__ unsigned long long s_pairs;
    __shared__ int s_base[kChunk / 32][kMaxRowGrid];       // per warp and row: slots before this warp's
    __shared__ unsigned s_mask[kChunk / 32][kMaxRowGrid + 1];  // per warp and row: the lanes covering it
    __shared__ int s_row0[kMaxRowGrid];                        // this chunk's start of each row
    const int lane = threadIdx.x & 31, wl = threadIdx.x >> 5;
    if (threadIdx.x == 0) s_pairs = 0;
    for (int r = threadIdx.x; r < kMaxRowGrid; r += kChunk) s_row0[r] = row0[(int64_t)r * n_chunks + blockIdx.x];
    unsigned *dif = s_mask[wl];
#pragma unroll
    for (int j = 0; j < 4; ++j) dif[lane + 32 * j] = 0u;
    if (lane == 0) dif[kMaxRowGrid] = 0u;
    __syncwarp();
    const int64_t j = (int64_t)blockIdx.x * kChunk + threadIdx.x;
    int i = 0, h = 0, k = 0;
    int4 bb = make_int4(0, 0, 0, 0);
    Grid gl = g;
    CullData d = {};
    if (j < n) {
        h = position_box<ITEMS>(bbox, tcount, order, j, g, t, i, k, gl, bb);
        if (h > 0) d = load_cull(rec, i);
    }
    // each row's covering lanes: every box's lane bit XORed in at its first row and out one past its
    // last, then the prefix XOR over the rows (4 rows a lane); their number
    if (h > 0) {
        atomicXor(&dif[bb.y], 1u << lane);
        atomicXor(&dif[bb.y + h], 1u << lane);
    }
    __syncwarp();
    {
        unsigned m[4];
#pragma unroll
        for (int jr = 0; jr < 4; ++jr) m[jr] = dif[4 * lane + jr] ^ (jr > 0 ? m[jr - 1] : 0u);
        unsigned x = m[3];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned y = __shfl_up_sync(kFullMask, x, o);
            if (lane >= o) x ^= y;
        }
        x ^= m[3];
        __syncwarp();
#pragma unroll
        for (int jr = 0; jr < 4; ++jr) {
            dif[4 * lane + jr] = m[jr] ^ x;
            s_base[wl][4 * lane + jr] = __popc(m[jr] ^ x);
        }
    }
    __syncthreads();
    // per row: the counts of the warps before each warp (exclusive prefix over the 8 warps)
    for (int r = threadIdx.x; r < kMaxRowGrid; r += kChunk) {
        int acc = 0;
#pragma unroll
        for (int w = 0; w < kChunk / 32; ++w) {
            const int c = s_base[w][r];
            s_base[w][r] = acc;
            acc += c;
        }
    }
    __syncthreads();
    const int incl = warp_incl_scan(h);
    const int rows = __shfl_sync(kFullMask, incl, 31);
    const int excl = incl - h;
    int kept = 0;
    for (int f0 = 0; f0 < rows; f0 += 32) {
        const int f = f0 + lane;
        const int p = lane_of(incl, f);
        const CullData e = shfl_cull(d, p);
        const int excl_p = __shfl_sync(kFullMask, excl, p);
        const int ty = __shfl_sync(kFullMask, bb.y, p) + f - excl_p;
        const int x0 = __shfl_sync(kFullMask, bb.x, p), x1 = __shfl_sync(kFullMask, bb.z, p);
        const int i_p = __shfl_sync(kFullMask, i, p);
        Grid gp = g;
        uint32_t item = 0;
        if (ITEMS) {
            gp.W = __shfl_sync(kFullMask, gl.W, p);
            gp.H = __shfl_sync(kFullMask, gl.H, p);
            item = (uint32_t)__shfl_sync(kFullMask, k, p) << kSpanItemShift;
        }
        if (f < rows) {
            int ka = 0, kb = -1;
            const int c = row_span_in_box(e, gp, ty, x0, x1, ka, kb);
            const int64_t s = (int64_t)s_row0[ty] + s_base[wl][ty] + __popc(s_mask[wl][ty] & ((1u << p) - 1u));
            if (s < ns_cap) {
                span_key[s] = c > 0 ? item | ((uint32_t)c << 15) | ((uint32_t)ka << 8) | (uint32_t)ty : kRowNone;
                span_prim[s] = (uint32_t)i_p;
            }
            kept += c;
        }
    }
    if (pair_total) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) kept += __shfl_xor_sync(kFullMask, kept, o);
        if (lane == 0 && kept) atomicAdd(&s_pairs, (unsigned long long)kept);
        __syncthreads();
        if (threadIdx.x == 0 && s_pairs) atomicAdd(pair_total, s_pairs);
    }
}

__device__ __forceinline__ int span_len(uint32_t key) { return (int)((key >> 15) & 0xffu); }

constexpr int kColPairs = 3968;                     // pairs per window of the column scatter
constexpr int kColStage = kColPairs + kMaxRowGrid;  // a window's pairs (its last span may run past it): 4096
constexpr int kColWarps = 8;

constexpr int kColSub = kColPairs / kColWarps;      // pairs per warp's share of a window: 496

// Window b of the column scatter holds the spans whose first pair lies in [b P, b P + P), P = 3968,
// and its warp w those whose first pair lies in sub-window u = 8 b + w, [u Q, u Q + Q), Q = 496:
// first[u] = the first span at or past u Q, first[8 nb] = ns.  The scan of the span lengths fills
// it as its epilogue: span j (first pair ex, v pairs) starts sub-window u = (ex + v) / Q at j + 1
// when u Q lies in (ex, ex + v] (every span holds at most 128 < Q pairs, so at most one such u); the
// sub-windows past the last pair start at ns.  Entries at or past cap are not written (the scan may
// run before the pair total is checked against the workspace).
struct ColFirstPost {
    int32_t *first;
    int64_t cap;
    __device__ __forceinline__ void operator()(int64_t j, int64_t ex, int32_t v) const {
        // 32-bit arithmetic: the pair offsets stay below 2^31 (checked before the pairs are placed)
        const uint32_t e = (uint32_t)ex, u = (e + (uint32_t)v) / (uint32_t)kColSub;
        if (u * (uint32_t)kColSub > e && (int64_t)u < cap) first[u] = (int32_t)(j + 1);
    }
    __device__ __forceinline__ void finish(int64_t ns, int64_t ni) const {
        const int64_t nsub = (ni + kColPairs - 1) / kColPairs * kColWarps;
        if (cap > 0) first[0] = 0;
        for (int64_t u = ni / kColSub + 1; u <= nsub && u < cap; ++u) first[u] = (int32_t)ns;
    }
};

// Column coverage of the spans [q0, q1) into d[0..128] as a difference array (+1 at the first kept
// column, -1 one past the last): its prefix over the columns is the number of pairs per column.
__device__ __forceinline__ void add_span_columns(const uint32_t *__restrict__ skey, int64_t q0, int64_t q1, int step,
                                                 int lane0, int *d) {
    for (int64_t q = q0 + lane0; q < q1; q += step) {
        const uint32_t key = skey[q];
        const int c = span_len(key);
        if (c > 0) {
            const int ka = (int)((key >> 8) & 0x7fu);
            atomicAdd(&d[ka], 1);
            atomicAdd(&d[ka + c], -1);
        }
    }
}

// In place: the inclusive prefix of d[0..127] over the columns, by one warp (4 columns a lane).
__device__ __forceinline__ void warp_column_prefix(int *d) {
    const int lane = threadIdx.x & 31;
    int v[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) v[j] = d[4 * lane + j] + (j > 0 ? v[j - 1] : 0);
    const int ex = warp_incl_scan(v[3]) - v[3];
    __syncwarp();
#pragma unroll
    for (int j = 0; j < 4; ++j) d[4 * lane + j] = ex + v[j];
    __syncwarp();
}

// hist[tx * nb + b] = the pairs of column tx among window b's spans (tx < ncol), one warp a window.
__global__ void __launch_bounds__(256) col_hist_kernel(const uint32_t *__restrict__ skey,
                                                       const int32_t *__restrict__ first, int64_t nb, int ncol,
                                                       int32_t *__restrict__ hist) {
    grid_dep_wait();
    __shared__ int d[kColWarps][kMaxRowGrid + 1];
    const int lane = threadIdx.x & 31, wl = threadIdx.x >> 5;
    const int64_t b = (int64_t)blockIdx.x * kColWarps + wl;
#pragma unroll
    for (int j = 0; j < 4; ++j) d[wl][lane + 32 * j] = 0;
    if (lane == 0) d[wl][kMaxRowGrid] = 0;
    __syncwarp();
    if (b < nb) add_span_columns(skey, first[b * kColWarps], first[(b + 1) * kColWarps], 32, lane, d[wl]);
    __syncwarp();
    warp_column_prefix(d[wl]);
    if (b < nb)
        for (int tx = lane; tx < ncol; tx += 32) hist[(int64_t)tx * nb + b] = d[wl][tx];
}

// The stable pass by column over the row-grouped spans, without expanding them first: block b
// places the pairs of its spans (the window of col_first_kernel) at off[tx * nb + b] (the scanned
// column-major histogram) plus their rank among the block's pairs of column tx.  Warp w takes the
// spans of sub-window 8 b + w (about 496 pairs each); a warp's counts per column (difference
// arrays) give every warp its start in each column.  A warp then takes its spans 32 at a time: each span's lane bit is
// XORed in at its first kept column and out one past its last, so the prefix XOR over the columns
// is, per column, the mask of the spans covering it; each lane walks an equal share of the 32 spans'
// pairs in order and ranks pair (span s, column tx) by the covering spans before s.  The pairs are
// staged in shared memory in output order (tile code and record in one word) and written out
// coalesced, with the tile code's range bounds where the code changes (by_code: x the least
// position, y the complement of the greatest end, both as unsigned minima over 0xffffffff-filled
// entries).
__global__ void __launch_bounds__(256) col_scatter_kernel(const uint32_t *__restrict__ skey,
                                                          const uint32_t *__restrict__ sprim,
                                                          const int32_t *__restrict__ first, int64_t nb, int ncol,
                                                          const int32_t *__restrict__ off,
                                                          uint32_t *__restrict__ vals, uint2 *__restrict__ by_code) {
    grid_dep_wait();
    __shared__ __align__(16) uint2 s_pc[kColStage];      // staged pairs: (tile code, record)
    __shared__ int s_base[kColWarps][kMaxRowGrid + 1];  // per warp and column: counts; then the XOR differences
    __shared__ uint2 s_mb[kColWarps][kMaxRowGrid];      // per warp and column: (covering spans, next place)
    __shared__ uint2 s_sp[kColWarps][32];               // per warp: the 32 spans' (first code | length << 24, record)
    __shared__ int s_gofs[kMaxRowGrid];                 // per column: output position minus staged position
    __shared__ int s_wsum[4];
    __shared__ int s_total;
    const int lane = threadIdx.x & 31, wl = threadIdx.x >> 5;
    for (int x = threadIdx.x; x < kColWarps * (kMaxRowGrid + 1); x += blockDim.x) (&s_base[0][0])[x] = 0;
    const int64_t wq0 = first[blockIdx.x * kColWarps + wl], wq1 = first[blockIdx.x * kColWarps + wl + 1];
    __syncthreads();
    add_span_columns(skey, wq0, wq1, 32, lane, s_base[wl]);
    __syncwarp();
    warp_column_prefix(s_base[wl]);
    __syncthreads();
    // per column: the warps' exclusive prefix, then the columns' starts in the staged order
    int ctot = 0;
    if (threadIdx.x < kMaxRowGrid) {
        const int tx = threadIdx.x;
#pragma unroll
        for (int w = 0; w < kColWarps; ++w) {
            const int c = s_base[w][tx];
            s_base[w][tx] = ctot;
            ctot += c;
        }
        const int incl = warp_incl_scan(ctot);
        if (lane == 31) s_wsum[wl] = incl;
        s_gofs[tx] = incl - ctot;  // exclusive within the warp for now
    }
    __syncthreads();
    if (threadIdx.x < kMaxRowGrid) {
        const int tx = threadIdx.x;
        int pre = 0;
        for (int w = 0; w < wl; ++w) pre += s_wsum[w];
        const int start = pre + s_gofs[tx];
#pragma unroll
        for (int w = 0; w < kColWarps; ++w) s_base[w][tx] += start;
        s_gofs[tx] = tx < ncol ? off[(int64_t)tx * nb + blockIdx.x] - start : 0;
        if (tx == kMaxRowGrid - 1) s_total = start + ctot;
    }
    __syncthreads();
    // this lane's columns 4 lane .. 4 lane + 3: the warp's next staged place in each
    int next[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) next[j] = s_base[wl][4 * lane + j];
    int *dif = s_base[wl];
    for (int64_t r0 = wq0; r0 < wq1; r0 += 32) {
        const int64_t q = r0 + lane;
        int len = 0, ka = 0;
        uint32_t code0 = 0, prim = 0;
        if (q < wq1) {
            const uint32_t key = skey[q];
            len = span_len(key);
            if (len > 0) {  // item, first kept column, row
                ka = (int)((key >> 8) & 0x7fu);
                code0 = ((key >> kSpanItemShift) << kItemShift) | ((uint32_t)ka << 7) | (key & 0x7fu);
                prim = sprim[q];
            }
        }
        const int incl = warp_incl_scan(len);
        const int total = __shfl_sync(kFullMask, incl, 31);
        __syncwarp();  // the previous round's readers are done with dif, s_mb and s_sp
        s_sp[wl][lane] = make_uint2(code0 | ((uint32_t)len << 24), prim);
#pragma unroll
        for (int j = 0; j < 4; ++j) dif[lane + 32 * j] = 0;
        if (lane == 0) dif[kMaxRowGrid] = 0;
        __syncwarp();
        if (len > 0) {
            atomicXor(&dif[ka], 1 << lane);
            atomicXor(&dif[ka + len], 1 << lane);
        }
        __syncwarp();
        unsigned m[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) m[j] = (unsigned)dif[4 * lane + j] ^ (j > 0 ? m[j - 1] : 0u);
        unsigned x = m[3];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned y = __shfl_up_sync(kFullMask, x, o);
            if (lane >= o) x ^= y;
        }
        x ^= m[3];  // the columns before this lane's
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            m[j] ^= x;
            s_mb[wl][4 * lane + j] = make_uint2(m[j], (unsigned)next[j]);
            next[j] += __popc(m[j]);
        }
        // this lane's share of the pairs: [k, kend) of the 32 spans' flattened list
        int k = (total * lane) >> 5;
        const int kend = (total * (lane + 1)) >> 5;
        int sp = lane_of(incl, k);
        int d = k - (__shfl_sync(kFullMask, incl, sp) - __shfl_sync(kFullMask, len, sp));
        __syncwarp();
        if (k < kend) {
            uint2 e = s_sp[wl][sp];
            int len_sp = (int)(e.x >> 24);
            for (; k < kend; ++k, ++d) {
                while (d == len_sp) {  // on to the next non-empty span
                    e = s_sp[wl][++sp];
                    len_sp = (int)(e.x >> 24);
                    d = 0;
                }
                const uint32_t code = (e.x & 0xffffffu) + ((uint32_t)d << 7);
                const uint2 mb = s_mb[wl][(code >> 7) & 0x7fu];
                s_pc[mb.y + __popc(mb.x & ((1u << sp) - 1u))] = make_uint2(code, e.y);
            }
        }
    }
    __syncthreads();
    // two staged pairs a thread: (code, record) of pairs li and li + 1 in one 16-byte read, the
    // neighbouring codes from the adjacent lanes
    const int T = s_total;
    const uint4 *s_pc2 = reinterpret_cast<const uint4 *>(s_pc);
    for (int base = 0; base < T; base += 2 * blockDim.x) {
        const int li = base + 2 * threadIdx.x;
        const uint4 e = li < T ? s_pc2[li >> 1] : make_uint4(0u, 0u, 0u, 0u);
        uint32_t prev = __shfl_up_sync(kFullMask, e.z, 1);
        uint32_t next = __shfl_down_sync(kFullMask, e.x, 1);
        if (li >= T) continue;
        if (lane == 0) prev = li > 0 ? s_pc[li - 1].x : ~e.x;
        if (li + 2 >= T) next = ~e.z;
        else if (lane == 31) next = s_pc[li + 2].x;
        const uint32_t g0 = (uint32_t)(s_gofs[(e.x >> 7) & 0x7fu] + li);
        vals[g0] = e.y;
        if (prev != e.x) atomicMin(&by_code[e.x].x, g0);
        if (li + 1 < T) {
            const uint32_t g1 = (uint32_t)(s_gofs[(e.z >> 7) & 0x7fu] + li + 1);
            vals[g1] = e.w;
            if (e.z != e.x) {
                atomicMin(&by_code[e.x].y, ~(g0 + 1u));
                atomicMin(&by_code[e.z].x, g1);
            }
            if (next != e.z) atomicMin(&by_code[e.z].y, ~(g1 + 1u));
        } else {
            atomicMin(&by_code[e.x].y, ~(g0 + 1u));
        }
    }
}

struct SpanLenItem {  // scan items: the pairs of row-grouped span q
    const uint32_t *skey;
    __device__ __forceinline__ int32_t operator()(int64_t q) const { return span_len(skey[q]); }
};

// ranges[tile0[k] + ty Wt[k] + tx] = the range found for tile code (k << 14) | (tx << 7) | ty
// (by_code as the column scatter leaves it: [x, ~y), x = 0xffffffff for a code with no pair)
__global__ void permute_ranges_kernel(const uint2 *__restrict__ by_code, RowItems t, int64_t n_tiles,
                                      int2 *__restrict__ ranges) {
    grid_dep_wait();
    const int64_t gt = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (gt >= n_tiles) return;
    int k = 0;
    while (k + 1 < t.count && gt >= t.tile0[k + 1]) ++k;
    const int local = (int)(gt - t.tile0[k]);
    const int tx = local % t.Wt[k], ty = local / t.Wt[k];
    const uint2 r = by_code[((int64_t)k << kItemShift) | (tx << 7) | ty];
    ranges[gt] = r.x == 0xffffffffu ? make_int2(0, 0) : make_int2((int)r.x, (int)~r.y);
}

size_t align_up(size_t x) { return (x + 255) / 256 * 256; }

// Tile codes a table can produce: (count - 1) << 14 plus the widest grid's (tx << 7) | ty.
int64_t n_codes(const RowItems &t) {
    int wt = 1;
    for (int k = 0; k < t.count; ++k) wt = t.Wt[k] > wt ? t.Wt[k] : wt;
    return ((int64_t)(t.count - 1) << kItemShift) + (int64_t)wt * kMaxRowGrid;
}

// The widest grid's tile columns: the columns of the column scatter's histogram.
int n_columns(const RowItems &t) {
    int wt = 1;
    for (int k = 0; k < t.count; ++k) wt = t.Wt[k] > wt ? t.Wt[k] : wt;
    return wt;
}

int64_t col_blocks(int64_t ni) { return (ni + kColPairs - 1) / kColPairs; }

// The row-count matrix (128 rows x chunks of 256 positions) and its scan depend on the records only;
// a span slot costs 12 bytes (key, record, pair offset); the pairs need the column histogram (one
// count per column and window of 3968 pairs) and its scan.
struct RowsLayout {
    size_t count, row0, part_n, totals;   // depend on the records only
    size_t skey, sprim, pair0, part_s;    // on the span slots
    size_t first, hist, off, part_h;      // on the pairs
    size_t by_code;
    size_t total;
};

int64_t row_count_entries(int64_t n) { return (int64_t)kMaxRowGrid * ((n + kChunk - 1) / kChunk); }

RowsLayout rows_layout(int64_t n, int64_t ns, int64_t ni, const RowItems &t) {
    RowsLayout L;
    size_t o = 0;
    auto take = [&](size_t bytes) {
        const size_t at = o;
        o += align_up(bytes);
        return at;
    };
    const int64_t nc = n_codes(t), m = row_count_entries(n);
    L.count = take((size_t)m * 4);
    L.row0 = take((size_t)(m + 1) * 4);
    L.part_n = take(scan_partials_bytes(m > n ? m : n));  // the row-count scan, then the kept-count sum
    L.totals = take(4 * sizeof(int64_t));
    L.skey = take((size_t)ns * 4);
    L.sprim = take((size_t)ns * 4);
    L.pair0 = take((size_t)(ns + 1) * 4);
    L.part_s = take(scan_partials_bytes(ns));
    const int64_t nb = col_blocks(ni), mh = nb * n_columns(t);
    L.first = take((size_t)(nb * kColWarps + 1) * 4);
    L.hist = take((size_t)mh * 4);
    L.off = take((size_t)(mh + 1) * 4);
    L.part_h = take(scan_partials_bytes(mh));
    L.by_code = take((size_t)nc * 8);
    L.total = o;
    return L;
}

}  // namespace

RowItems row_items_views(const XprCamera &cam, const XprConfig &cfg, int64_t n, int n_views) {
    RowItems t;
    memset(&t, 0, sizeof(t));
    t.count = n_views;
    const int Wt = tiles_x(cam, cfg), Ht = tiles_y(cam, cfg);
    for (int v = 0; v <= n_views; ++v) {
        t.rec0[v] = (int64_t)v * n;
        t.tile0[v] = (int64_t)v * Wt * Ht;
    }
    for (int v = 0; v < n_views; ++v) {
        t.W[v] = cam.width;
        t.H[v] = cam.height;
        t.Wt[v] = Wt;
        t.Ht[v] = Ht;
    }
    return t;
}

RowItems row_items_items(const XprCamera *cams, const XprItem *items, int n_items, const XprConfig &cfg) {
    RowItems t;
    memset(&t, 0, sizeof(t));
    t.count = n_items;
    int64_t tile = 0;
    for (int k = 0; k < n_items; ++k) {
        t.rec0[k] = items[k].rec_offset;
        t.tile0[k] = tile;
        t.W[k] = cams[k].width;
        t.H[k] = cams[k].height;
        t.Wt[k] = tiles_x(cams[k], cfg);
        t.Ht[k] = tiles_y(cams[k], cfg);
        tile += (int64_t)t.Wt[k] * t.Ht[k];
    }
    t.rec0[n_items] = n_items > 0 ? items[n_items - 1].rec_offset + (items[n_items - 1].n + 31) / 32 * 32 : 0;
    t.tile0[n_items] = tile;
    return t;
}

bool bin_rows_supported(const XprCamera &cam, const XprConfig &cfg) {
    return tiles_x(cam, cfg) <= kMaxRowGrid && tiles_y(cam, cfg) <= kMaxRowGrid;
}

bool bin_rows_supported(const RowItems &t) {
    if (t.count < 1 || t.count > kMaxItems) return false;
    for (int k = 0; k < t.count; ++k)
        if (t.Wt[k] > kMaxRowGrid || t.Ht[k] > kMaxRowGrid) return false;
    return true;
}

size_t bin_rows_workspace_bytes(int64_t n_records, int64_t n_spans, int64_t n_isect, const RowItems &t) {
    return rows_layout(n_records, n_spans, n_isect, t).total;
}

namespace {

// The largest span-slot room the workspace holds beside room for `capacity` pairs (-1: none).
int64_t span_room(int64_t n, int64_t capacity, const RowItems &t, size_t ws_bytes) {
    if (rows_layout(n, 0, capacity, t).total > ws_bytes) return -1;
    int64_t lo = 0, hi = 0x7fffffffLL;
    while (lo < hi) {
        const int64_t mid = lo + (hi - lo + 1) / 2;
        if (rows_layout(n, mid, capacity, t).total <= ws_bytes) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// Per host thread and device: a page-locked buffer for the counts the binning reads back and two
// events that mark when each count has landed, so the host waits on a count while the kernels
// that do not need it are already queued behind it.  NULL when they cannot be created.
struct Readback {
    int64_t *host = nullptr;
    cudaEvent_t ev[2] = {nullptr, nullptr};
};

Readback *readback_slots() {
    constexpr int kDevices = 64;
    thread_local Readback r[kDevices];
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kDevices) {
        cudaGetLastError();
        return nullptr;
    }
    Readback &s = r[dev];
    if (!s.host) {
        void *h = nullptr;
        if (cudaHostAlloc(&h, 64, cudaHostAllocDefault) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        for (auto &e : s.ev)
            if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) {
                cudaGetLastError();
                return nullptr;  // the buffer stays for the next attempt
            }
        s.host = reinterpret_cast<int64_t *>(h);
    }
    return &s;
}

}  // namespace

// order: the depth order of the n records (each item's in its own block); isect_count (NULL: none):
// their kept tile counts.  The span total (and, with isect_count, the pair total) is read back
// after the scan of the row-count matrix, the pair total otherwise from the emission.  When the
// workspace has room for `capacity` pairs and some span slots, the emission is queued before the
// host reads the span total (its writes bounded by that room) and the span-length scan before it
// reads the pair total, so the device does not idle while the host waits; otherwise each count is read
// with the stream synchronised before the work that needs it.  Returns XPR_ERR_CAPACITY (n_isect
// and n_spans set as far as known, vals and ranges unwritten) when vals holds fewer than n_isect
// pairs or the workspace is below bin_rows_workspace_bytes.
int launch_bin_rows(const float *rec, const int32_t *bbox, const int32_t *tc, const int32_t *isect_count,
                    const int32_t *order, int64_t n, const RowItems &t, const XprConfig &cfg, int32_t *ranges,
                    uint32_t *vals, int64_t capacity, int64_t *n_isect, int64_t *n_spans, void *ws, size_t ws_bytes,
                    cudaStream_t st) {
    if (!bin_rows_supported(t))
        return fail(XPR_ERR_INVALID, "xpr_bin_rows: %d items, or a tile grid with more than 128 tile columns or rows",
                    t.count);
    Grid g;
    g.W = t.W[0];
    g.H = t.H[0];
    g.tw = cfg.tile_w;
    g.th = cfg.tile_h;
    g.Wt = t.Wt[0];
    g.Ht = t.Ht[0];
    g.ext = cfg.method == XPR_METHOD_3DGUT ? 1 : 0;
    const bool items = t.count > 1;
    const int64_t T = t.tile0[t.count];
    *n_isect = 0;
    *n_spans = 0;
    if (n == 0) {
        if (T > 0) XPR_CUDA_TRY(cudaMemsetAsync(ranges, 0, (size_t)T * 8, st));
        return XPR_OK;
    }
    const RowsLayout L0 = rows_layout(n, 0, 0, t);
    if (ws_bytes < L0.total) return fail(XPR_ERR_INVALID, "xpr_bin_rows: workspace %zu < %zu bytes", ws_bytes, L0.total);
    char *p = reinterpret_cast<char *>(ws);
    int32_t *count = reinterpret_cast<int32_t *>(p + L0.count);
    int32_t *row0 = reinterpret_cast<int32_t *>(p + L0.row0);
    int64_t *tot = reinterpret_cast<int64_t *>(p + L0.totals);  // span total, kept total, pair total, emitted pairs
    const int4 *bb4 = reinterpret_cast<const int4 *>(bbox);
    const int64_t ns_cap = span_room(n, capacity, t, ws_bytes);
    Readback *rb = ns_cap >= 0 ? readback_slots() : nullptr;
    // the slots grouped by row: the box rows counted per (row, chunk of 256 depth positions), the
    // row-major matrix scanned into each chunk's start in each row (its total: the slot count);
    // with the kept counts, the pair total is their sum
    const int64_t n_chunks = (n + kChunk - 1) / kChunk;
    XPR_CUDA_TRY(launch_dependent(items ? row_count_kernel<true> : row_count_kernel<false>, dim3((unsigned)n_chunks),
                                  dim3(kChunk), 0, st, bb4, tc, order, n, g, t, n_chunks, count));
    XPR_LAUNCH_CHECK("row_count_kernel");
    int s = launch_scan(CountItem{count}, row0, row_count_entries(n), p + L0.part_n, tot, st);
    if (s != XPR_OK) return s;
    if (isect_count) {
        s = launch_scan(CountItem{isect_count}, nullptr, n, p + L0.part_n, tot + 1, st);
        if (s != XPR_OK) return s;
    } else if (rb) {
        XPR_CUDA_TRY(cudaMemsetAsync(tot + 3, 0, sizeof(int64_t), st));
    }
    auto emit = [&](const RowsLayout &L, int64_t room, unsigned long long *pairs) -> int {
        uint32_t *skey = reinterpret_cast<uint32_t *>(p + L.skey), *sprim = reinterpret_cast<uint32_t *>(p + L.sprim);
        XPR_CUDA_TRY(launch_dependent(items ? span_emit_kernel<true> : span_emit_kernel<false>,
                                      dim3((unsigned)n_chunks), dim3(kChunk), 0, st, rec, bb4, tc, order, n, g, t,
                                      n_chunks, (const int32_t *)row0, room, skey, sprim, pairs));
        XPR_LAUNCH_CHECK("span_emit_kernel");
        return XPR_OK;
    };
    int64_t ns = 0, ni = 0;
    RowsLayout L;
    bool early = rb != nullptr;
    if (early) {
        L = rows_layout(n, ns_cap, capacity, t);
        XPR_CUDA_TRY(cudaMemcpyAsync(rb->host, tot, 2 * sizeof(int64_t), cudaMemcpyDeviceToHost, st));
        XPR_CUDA_TRY(cudaEventRecord(rb->ev[0], st));
        if ((s = emit(L, ns_cap, isect_count ? nullptr : reinterpret_cast<unsigned long long *>(tot + 3)))) return s;
        if (!isect_count) {
            XPR_CUDA_TRY(cudaMemcpyAsync(rb->host + 2, tot + 3, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
            XPR_CUDA_TRY(cudaEventRecord(rb->ev[1], st));
        }
        XPR_CUDA_TRY(cudaEventSynchronize(rb->ev[0]));
        ns = rb->host[0];
        ni = isect_count ? rb->host[1] : 0;
    } else {
        int64_t h_tot[2] = {0, 0};
        XPR_CUDA_TRY(cudaMemcpyAsync(h_tot, tot, (isect_count ? 2 : 1) * sizeof(int64_t), cudaMemcpyDeviceToHost, st));
        XPR_CUDA_TRY(cudaStreamSynchronize(st));
        ns = h_tot[0];
        ni = isect_count ? h_tot[1] : 0;
    }
    *n_spans = ns;
    if (isect_count) *n_isect = ni;
    if (ns > 0x7fffffffLL || ni > 0x7fffffffLL)
        return fail(XPR_ERR_CAPACITY, "xpr_bin_rows: more than 2^31 - 1 spans or pairs");
    // the spans outgrew the room (or the pairs the capacity): on as if nothing had been queued
    // early (the emission again, into the regions this count fixes), so that the counts reported
    // are those of the synchronised protocol
    if (early && (ns > ns_cap || (isect_count && ni > capacity))) early = false;
    if (!early) {
        // without the kept counts the pair total is known only once the spans exist: the span
        // phase is checked here (its regions do not depend on the pair count) and the pair phase after
        L = rows_layout(n, ns, ni, t);
        if ((isect_count && ni > capacity) || ws_bytes < L.total) return XPR_ERR_CAPACITY;
        if ((s = emit(L, ns, nullptr))) return s;
    }
    uint32_t *skey = reinterpret_cast<uint32_t *>(p + L.skey), *sprim = reinterpret_cast<uint32_t *>(p + L.sprim);
    int32_t *pair0 = reinterpret_cast<int32_t *>(p + L.pair0);
    // the first pair of every span; the spans starting each sub-window of the column scatter (its
    // room: the region sized for the pairs when their count is known here, else what the workspace
    // leaves after its start)
    const int64_t first_cap = early || isect_count ? (int64_t)((L.hist - L.first) / 4)
                                                   : (int64_t)((ws_bytes - L.first) / 4);
    s = launch_scan(SpanLenItem{skey}, pair0, ns, p + L.part_s, tot + 2, st,
                    ColFirstPost{reinterpret_cast<int32_t *>(p + L.first), first_cap});
    if (s != XPR_OK) return s;
    if (!isect_count) {
        if (early) {
            XPR_CUDA_TRY(cudaEventSynchronize(rb->ev[1]));
            ni = rb->host[2];
        } else {
            XPR_CUDA_TRY(cudaMemcpyAsync(&ni, tot + 2, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
            XPR_CUDA_TRY(cudaStreamSynchronize(st));
        }
        *n_isect = ni;
        if (ni > 0x7fffffffLL) return fail(XPR_ERR_CAPACITY, "xpr_bin_rows: more than 2^31 - 1 pairs");
        if (ni > capacity || (!early && ws_bytes < rows_layout(n, ns, ni, t).total)) return XPR_ERR_CAPACITY;
    }
    const RowsLayout LP = early ? L : rows_layout(n, ns, ni, t);
    // the pass by column straight from the spans: windows of 3968 pairs, their column histogram
    // scanned column-major, each window's pairs placed by column and rank
    uint2 *by_code = reinterpret_cast<uint2 *>(p + LP.by_code);
    XPR_CUDA_TRY(cudaMemsetAsync(by_code, 0xff, (size_t)n_codes(t) * 8, st));
    if (ni > 0) {
        const int64_t nb = col_blocks(ni);
        const int ncol = n_columns(t);
        const int32_t *first = reinterpret_cast<const int32_t *>(p + LP.first);
        int32_t *hist = reinterpret_cast<int32_t *>(p + LP.hist), *off = reinterpret_cast<int32_t *>(p + LP.off);
        XPR_CUDA_TRY(launch_dependent(col_hist_kernel, dim3((unsigned)((nb + kColWarps - 1) / kColWarps)),
                                      dim3(256), 0, st, (const uint32_t *)skey, first, nb, ncol, hist));
        XPR_LAUNCH_CHECK("col_hist_kernel");
        s = launch_scan(CountItem{hist}, off, nb * ncol, p + LP.part_h, nullptr, st);
        if (s != XPR_OK) return s;
        XPR_CUDA_TRY(launch_dependent(col_scatter_kernel, dim3((unsigned)nb), dim3(256), 0, st, (const uint32_t *)skey,
                                      (const uint32_t *)sprim, first, nb, ncol, (const int32_t *)off,
                                      vals, by_code));
        XPR_LAUNCH_CHECK("col_scatter_kernel");
    }
    if (T > 0) {
        XPR_CUDA_TRY(launch_dependent(permute_ranges_kernel, dim3((unsigned)((T + 255) / 256)), dim3(256), 0, st,
                                      (const uint2 *)by_code, t, T, reinterpret_cast<int2 *>(ranges)));
        XPR_LAUNCH_CHECK("permute_ranges_kernel");
    }
    return XPR_OK;
}

}  // namespace xpr
