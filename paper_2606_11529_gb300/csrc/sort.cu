// Rasterizer, second half (Sec. 4.2 "Sort and identify bounds"): stable LSD radix sort of the
// intersection pairs by tile (and depth), then the per-tile segment bounds [start, end).
//
// Keys are either u64 (tile << 32 | depth bits; xpr_sort) or u32 tile ids (xpr_sort_tiles, for
// pairs emitted in depth order, where a stable sort by tile alone gives the (tile, depth) order).
// Each 8-bit pass is reduce-then-scan over tiles of 4096 keys:
//   * the histogram kernel counts the tile's digits (each thread 16 consecutive keys read as
//     vectors, equal neighbouring digits added as one run) into a block-major (tile x digit)
//     matrix, one coalesced row per tile;
//   * a column scan of that matrix (32-row segment sums, a scan over segments per digit, then the
//     in-place prefix) turns every entry into the global output offset of the tile's digit run,
//     the digits in order and the tiles in order within a digit;
//   * the scatter kernel ranks its keys stably (warp w owns a contiguous run of 512 keys visited in
//     index order, __match_any_sync groups equal digits within each round of 32), places every key
//     at its rank in a block-local sorted copy in shared memory, and writes the copy out in order,
//     so consecutive threads write consecutive addresses of one digit's output run.
// The segment bounds come from one pass over the sorted keys (a boundary wherever neighbouring
// keys differ in tile).
#include "xpr_internal.cuh"

namespace xpr {
namespace {

constexpr int kThreads = 256;
constexpr int kItems = 16;
constexpr int kWarps = kThreads / 32;
constexpr int kWarpKeys = 32 * kItems;    // 512
constexpr int kTile = kThreads * kItems;  // 4096
constexpr int kRadix = 256;
constexpr int kSegRows = 32;              // matrix rows per segment of the column scan
constexpr int kRangeItems = 8;            // keys per thread of the segment-bound kernel

template <typename K>
constexpr size_t scatter_smem() {
    return (size_t)kTile * sizeof(K) + (size_t)kTile * 4 + (size_t)kWarps * kRadix * 4 + 2 * (size_t)kRadix * 4 + 64;
}

template <typename K>
__device__ __forceinline__ uint32_t tile_of(K key);
template <>
__device__ __forceinline__ uint32_t tile_of<uint64_t>(uint64_t key) {
    return (uint32_t)(key >> 32);
}
template <>
__device__ __forceinline__ uint32_t tile_of<uint32_t>(uint32_t key) {
    return key;
}

// Loads keys [i, i + 4) (16-byte aligned) of a u32 or u64 array.
__device__ __forceinline__ void load4(const uint32_t *p, int64_t i, uint32_t (&k)[4]) {
    const uint4 v = *reinterpret_cast<const uint4 *>(p + i);
    k[0] = v.x;
    k[1] = v.y;
    k[2] = v.z;
    k[3] = v.w;
}
__device__ __forceinline__ void load4(const uint64_t *p, int64_t i, uint64_t (&k)[4]) {
    const ulonglong2 a = *reinterpret_cast<const ulonglong2 *>(p + i);
    const ulonglong2 b = *reinterpret_cast<const ulonglong2 *>(p + i + 2);
    k[0] = a.x;
    k[1] = a.y;
    k[2] = b.x;
    k[3] = b.y;
}

// hist[b][d] = number of keys of tile b with digit d.  vec: kin is 16-byte aligned.
template <typename K>
__global__ void __launch_bounds__(kThreads) radix_hist_kernel(const K *__restrict__ kin, int64_t n, int shift,
                                                              uint32_t mask, int32_t *__restrict__ hist, bool vec) {
    __shared__ int s[kWarps][kRadix];
    for (int d = threadIdx.x; d < kWarps * kRadix; d += kThreads) (&s[0][0])[d] = 0;
    __syncthreads();
    const int w = threadIdx.x >> 5;
    const int64_t base = (int64_t)blockIdx.x * kTile + (int64_t)threadIdx.x * kItems;
    int prev = -1, run = 0;
    auto add = [&](K key) {
        const int d = (int)((uint32_t)(key >> shift) & mask);
        if (d == prev) {
            ++run;
        } else {
            if (run) atomicAdd(&s[w][prev], run);
            prev = d;
            run = 1;
        }
    };
    if (vec && base + kItems <= n) {
#pragma unroll
        for (int q = 0; q < kItems; q += 4) {
            K k[4];
            load4(kin, base + q, k);
#pragma unroll
            for (int r = 0; r < 4; ++r) add(k[r]);
        }
    } else {
        for (int q = 0; q < kItems; ++q)
            if (base + q < n) add(kin[base + q]);
    }
    if (run) atomicAdd(&s[w][prev], run);
    __syncthreads();
    int sum = 0;
#pragma unroll
    for (int ww = 0; ww < kWarps; ++ww) sum += s[ww][threadIdx.x];
    hist[(int64_t)blockIdx.x * kRadix + threadIdx.x] = sum;
}

// Column scan of the (tile x digit) matrix, step 1: part[g][d] = sum of rows [32 g, 32 g + 32).
__global__ void __launch_bounds__(kRadix) colsum_kernel(const int32_t *__restrict__ hist, int64_t nb,
                                                        int32_t *__restrict__ part) {
    const int64_t g = blockIdx.x;
    const int64_t r0 = g * kSegRows, r1 = min(r0 + kSegRows, nb);
    const int32_t *h = hist + r0 * kRadix + threadIdx.x;
    int sum = 0;
#pragma unroll 8
    for (int64_t r = r0; r < r1; ++r, h += kRadix) sum += *h;
    part[g * kRadix + threadIdx.x] = sum;
}

// Block-wide exclusive scan of one int per thread (blockDim.x a multiple of 32, <= 1024).
__device__ __forceinline__ int block_excl_scan(int v, int *s_warp, int *total) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) s_warp[wid] = x;
    __syncthreads();
    if (wid == 0) {
        int t = lane < nw ? s_warp[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += y;
        }
        if (lane < nw) s_warp[lane] = t;
    }
    __syncthreads();
    const int pre = wid > 0 ? s_warp[wid - 1] : 0;
    *total = s_warp[nw - 1];
    __syncthreads();
    return pre + x - v;
}

// Step 2, one block per digit d: exclusive prefix of part[.][d] over the segments (in place) and
// the digit's total.
__global__ void __launch_bounds__(1024) segscan_kernel(int32_t *__restrict__ part, int64_t nseg,
                                                       int32_t *__restrict__ dtot) {
    __shared__ int s_warp[32];
    const int d = blockIdx.x;
    int carry = 0;
    for (int64_t b0 = 0; b0 < nseg; b0 += blockDim.x) {
        const int64_t g = b0 + threadIdx.x;
        const int v = g < nseg ? part[g * kRadix + d] : 0;
        int tot;
        const int ex = block_excl_scan(v, s_warp, &tot);
        if (g < nseg) part[g * kRadix + d] = carry + ex;
        carry += tot;
    }
    if (threadIdx.x == 0) dtot[d] = carry;
}

// Step 3: hist[r][d] <- (keys of digits < d) + (keys of digit d in rows < r).
__global__ void __launch_bounds__(kRadix) colapply_kernel(int32_t *__restrict__ hist, int64_t nb,
                                                          const int32_t *__restrict__ part,
                                                          const int32_t *__restrict__ dtot) {
    __shared__ int s_warp[32];
    const int64_t g = blockIdx.x;
    const int d = threadIdx.x;
    int tot;
    int run = block_excl_scan(dtot[d], s_warp, &tot) + part[g * kRadix + d];
    const int64_t r0 = g * kSegRows, r1 = min(r0 + kSegRows, nb);
    int32_t *h = hist + r0 * kRadix + d;
    for (int64_t r = r0; r < r1; ++r, h += kRadix) {
        const int x = *h;
        *h = run;
        run += x;
    }
}

// Last pass only (ranges non-NULL): the output is in final order, and inside a block's local run
// the keys of one tile are contiguous (one digit group, ordered by the lower digits), so the
// first and last key of each local tile run give that tile's segment bounds through one atomic
// min / max each (ranges start as [INT_MAX, 0) and untouched tiles are reset to [0, 0) after).
// kout NULL: the sorted keys are not written (only their segment bounds are wanted).
template <typename K>
__global__ void __launch_bounds__(kThreads) radix_scatter_kernel(const K *__restrict__ kin,
                                                                 const uint32_t *__restrict__ vin,
                                                                 K *__restrict__ kout, uint32_t *__restrict__ vout,
                                                                 int64_t n, int shift, uint32_t mask,
                                                                 const int32_t *__restrict__ offs,
                                                                 int2 *__restrict__ ranges, uint32_t n_tiles) {
    extern __shared__ __align__(16) unsigned char smem[];
    K *s_key = reinterpret_cast<K *>(smem);
    uint32_t *s_val = reinterpret_cast<uint32_t *>(smem + (size_t)kTile * sizeof(K));
    int(*s_hist)[kRadix] = reinterpret_cast<int(*)[kRadix]>(smem + (size_t)kTile * (sizeof(K) + 4));
    int *s_start = reinterpret_cast<int *>(smem + (size_t)kTile * (sizeof(K) + 4) + (size_t)kWarps * kRadix * 4);
    int *s_gofs = s_start + kRadix;
    int *s_wsum = s_gofs + kRadix;  // kWarps partial sums for the digit scan

    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int d = threadIdx.x; d < kWarps * kRadix; d += kThreads) (&s_hist[0][0])[d] = 0;
    __syncthreads();
    const int64_t block_base = (int64_t)blockIdx.x * kTile;
    const K *kb = kin + block_base;
    const uint32_t *vb = vin + block_base;
    const int count = (int)min((int64_t)kTile, n - block_base);
    const int wbase = w * kWarpKeys;
    const unsigned lt_mask = (1u << lane) - 1u;
    // Lanes with equal digits are found with one ballot per digit bit (the match instruction runs
    // on a narrow pipe that limited this kernel); the group's lowest lane alone reads and bumps
    // the warp's running count of the digit and hands the old count to its group by a shuffle.
    const int nbits = __popc(mask);
    // all of the thread's keys (and, for 4-byte keys, values) are loaded before any ranking so
    // that a warp has kItems loads in flight instead of one per round
    constexpr bool kHoldVals = sizeof(K) == 4;
    K kreg[kItems];
    uint32_t vreg[kHoldVals ? kItems : 1];
#pragma unroll
    for (int r = 0; r < kItems; ++r) {
        const int idx = wbase + r * 32 + lane;
        kreg[r] = idx < count ? kb[idx] : K(0);
        if (kHoldVals) vreg[kHoldVals ? r : 0] = idx < count ? vb[idx] : 0u;
    }
    int dr[kItems];
#pragma unroll
    for (int r = 0; r < kItems; ++r) {
        const int idx = wbase + r * 32 + lane;
        const bool valid = idx < count;
        const uint32_t d = valid ? (uint32_t)(kreg[r] >> shift) & mask : 0u;
        unsigned peers = __ballot_sync(0xffffffffu, valid);
        for (int b = 0; b < nbits; ++b) {
            const bool bit = (d >> b) & 1u;
            const unsigned bal = __ballot_sync(0xffffffffu, bit);
            peers &= bit ? bal : ~bal;
        }
        const int leader = valid ? __ffs(peers) - 1 : lane;
        int cur = 0;
        if (valid && lane == leader) {
            cur = s_hist[w][d];
            s_hist[w][d] = cur + __popc(peers);
        }
        cur = __shfl_sync(0xffffffffu, cur, leader);
        __syncwarp();  // the next round's leaders read what this round's leaders wrote
        dr[r] = (int)(d << 16) | (cur + __popc(peers & lt_mask));
    }
    __syncthreads();
    // per digit: prefix over warps (in place) and the digit's total in this block
    const int d0 = threadIdx.x;
    int tot = 0;
#pragma unroll
    for (int ww = 0; ww < kWarps; ++ww) {
        const int c = s_hist[ww][d0];
        s_hist[ww][d0] = tot;
        tot += c;
    }
    // exclusive scan of the digit totals over the block -> start of each digit in the local order
    int x = tot;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) s_wsum[w] = x;
    __syncthreads();
    int wpre = 0;
    for (int ww = 0; ww < w; ++ww) wpre += s_wsum[ww];
    const int start = wpre + x - tot;
    s_start[d0] = start;
    s_gofs[d0] = offs[(int64_t)blockIdx.x * kRadix + d0] - start;
    __syncthreads();
    // place every key at its local rank
#pragma unroll
    for (int r = 0; r < kItems; ++r) {
        const int idx = wbase + r * 32 + lane;
        if (idx < count) {
            const int d = dr[r] >> 16;
            const int pos = s_start[d] + s_hist[w][d] + (dr[r] & 0xffff);
            s_key[pos] = kreg[r];
            s_val[pos] = kHoldVals ? vreg[kHoldVals ? r : 0] : vb[idx];
        }
    }
    __syncthreads();
    // write the block's sorted run: consecutive threads, consecutive output addresses within a digit
    for (int s = threadIdx.x; s < count; s += kThreads) {
        const K k = s_key[s];
        const int d = (int)((uint32_t)(k >> shift) & mask);
        const int64_t g = (int64_t)s_gofs[d] + s;
        if (kout) kout[g] = k;
        vout[g] = s_val[s];
        if (ranges) {
            const uint32_t t = tile_of<K>(k);
            if (t < n_tiles) {
                if (s == 0 || tile_of<K>(s_key[s - 1]) != t) atomicMin(&ranges[t].x, (int)g);
                if (s == count - 1 || tile_of<K>(s_key[s + 1]) != t) atomicMax(&ranges[t].y, (int)(g + 1));
            }
        }
    }
}

__global__ void init_ranges_kernel(int2 *__restrict__ ranges, int n_tiles) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n_tiles) ranges[t] = make_int2(0x7fffffff, 0);
}

__global__ void fix_empty_ranges_kernel(int2 *__restrict__ ranges, int n_tiles) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n_tiles && ranges[t].x == 0x7fffffff) ranges[t] = make_int2(0, 0);
}
// Segment bounds: thread t looks at keys [8t, 8t + 8) and the key before them; a tile starts
// where the tile differs from the previous key's and ends where it differs from the next key's.
// vec: keys is 16-byte aligned.  Empty tiles keep the [0, 0) the caller cleared.
template <typename K>
__global__ void __launch_bounds__(256) tile_ranges_kernel(const K *__restrict__ keys, int64_t n, uint32_t n_tiles,
                                                          int2 *__restrict__ ranges, bool vec) {
    const int64_t i0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * kRangeItems;
    if (i0 >= n) return;
    const int m = (int)min((int64_t)kRangeItems, n - i0);
    K a[4], b[4];
    if (vec && m == kRangeItems) {
        load4(keys, i0, a);
        load4(keys, i0 + 4, b);
    } else {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            a[q] = q < m ? keys[i0 + q] : K(0);
            b[q] = q + 4 < m ? keys[i0 + 4 + q] : K(0);
        }
    }
    uint32_t prev = i0 > 0 ? tile_of<K>(keys[i0 - 1]) : 0xffffffffu;
#pragma unroll
    for (int q = 0; q < kRangeItems; ++q) {
        const uint32_t t = tile_of<K>(q < 4 ? a[q] : b[q - 4]);
        if (q < m && t != prev) {
            if (t < n_tiles) ranges[t].x = (int)(i0 + q);
            if (prev < n_tiles) ranges[prev].y = (int)(i0 + q);
            prev = t;
        }
    }
    if (i0 + m == n && prev < n_tiles) ranges[prev].y = (int)n;
}

inline size_t align256(size_t b) { return (b + 255) / 256 * 256; }

int bits_for(int64_t x) {
    int b = 0;
    while (x > 0) {
        ++b;
        x >>= 1;
    }
    return b;
}

inline bool is_aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; }

template <typename K>
size_t workspace_bytes(int64_t n) {
    const int64_t nb = max((int64_t)1, (n + kTile - 1) / kTile);
    const int64_t nseg = (nb + kSegRows - 1) / kSegRows;
    return align256((size_t)n * sizeof(K)) + align256((size_t)n * 4) + align256((size_t)nb * kRadix * 4) +
           align256((size_t)nseg * kRadix * 4) + align256((size_t)kRadix * 4);
}

// Sorts (kin, vin) by key bits [begin_bit, end_bit) into (kout, vout), then finds tile ranges.
template <typename K>
int radix_sort(const K *keys_in, const uint32_t *vals_in, int64_t n, int32_t n_tiles, int begin_bit, int end_bit,
               K *keys_out, uint32_t *vals_out, int32_t *ranges, void *ws, size_t ws_bytes, cudaStream_t st) {
    XPR_CUDA_TRY(cudaMemsetAsync(ranges, 0, (size_t)n_tiles * 2 * sizeof(int32_t), st));
    if (n == 0) return XPR_OK;
    if (ws_bytes < workspace_bytes<K>(n))
        return fail(XPR_ERR_INVALID, "sort: workspace %zu bytes < required %zu", ws_bytes, workspace_bytes<K>(n));
    // the dynamic shared-memory limit is a per-function attribute of the current device's module
    // (one value per key type, so concurrent callers all set the same limit)
    XPR_CUDA_TRY(cudaFuncSetAttribute(radix_scatter_kernel<K>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)scatter_smem<K>()));
    const int64_t nb = (n + kTile - 1) / kTile;
    const int64_t nseg = (nb + kSegRows - 1) / kSegRows;
    char *p = reinterpret_cast<char *>(ws);
    K *alt_k = reinterpret_cast<K *>(p);
    p += align256((size_t)n * sizeof(K));
    uint32_t *alt_v = reinterpret_cast<uint32_t *>(p);
    p += align256((size_t)n * 4);
    int32_t *hist = reinterpret_cast<int32_t *>(p);
    p += align256((size_t)nb * kRadix * 4);
    int32_t *part = reinterpret_cast<int32_t *>(p);
    p += align256((size_t)nseg * kRadix * 4);
    int32_t *dtot = reinterpret_cast<int32_t *>(p);

    const int passes = begin_bit < end_bit ? (end_bit - begin_bit + 7) / 8 : 0;
    if (passes == 0) {
        if (keys_out)
            XPR_CUDA_TRY(cudaMemcpyAsync(keys_out, keys_in, (size_t)n * sizeof(K), cudaMemcpyDeviceToDevice, st));
        XPR_CUDA_TRY(cudaMemcpyAsync(vals_out, vals_in, (size_t)n * 4, cudaMemcpyDeviceToDevice, st));
    }
    const K *src_k = keys_in;
    const uint32_t *src_v = vals_in;
    int2 *rg = reinterpret_cast<int2 *>(ranges);
    const unsigned tgrid = (unsigned)((n_tiles + 255) / 256);
    if (passes > 0) {
        init_ranges_kernel<<<tgrid, 256, 0, st>>>(rg, n_tiles);
        XPR_LAUNCH_CHECK("init_ranges_kernel");
    }
    for (int pass = 0; pass < passes; ++pass) {
        const int shift = begin_bit + 8 * pass;
        const int nbits = min(8, end_bit - shift);
        const uint32_t mask = (1u << nbits) - 1u;
        const bool to_out = ((passes - 1 - pass) % 2) == 0;
        const bool last = pass == passes - 1;
        uint32_t *dst_v = to_out ? vals_out : alt_v;
        // keys: keys_out / alt ping-pong; without keys_out the last pass writes no keys and the
        // others alternate alt, keys_in (the caller's input doubles as the second buffer)
        K *dst_k = keys_out ? (to_out ? keys_out : alt_k)
                            : (last ? nullptr : ((pass % 2) == 0 ? alt_k : const_cast<K *>(keys_in)));
        radix_hist_kernel<K><<<(unsigned)nb, kThreads, 0, st>>>(src_k, n, shift, mask, hist, is_aligned16(src_k));
        XPR_LAUNCH_CHECK("radix_hist_kernel");
        colsum_kernel<<<(unsigned)nseg, kRadix, 0, st>>>(hist, nb, part);
        XPR_LAUNCH_CHECK("colsum_kernel");
        segscan_kernel<<<kRadix, 1024, 0, st>>>(part, nseg, dtot);
        XPR_LAUNCH_CHECK("segscan_kernel");
        colapply_kernel<<<(unsigned)nseg, kRadix, 0, st>>>(hist, nb, part, dtot);
        XPR_LAUNCH_CHECK("colapply_kernel");
        radix_scatter_kernel<K><<<(unsigned)nb, kThreads, scatter_smem<K>(), st>>>(
            src_k, src_v, dst_k, dst_v, n, shift, mask, hist, last ? rg : nullptr, (uint32_t)n_tiles);
        XPR_LAUNCH_CHECK("radix_scatter_kernel");
        src_k = dst_k;
        src_v = dst_v;
    }
    if (passes > 0) {
        fix_empty_ranges_kernel<<<tgrid, 256, 0, st>>>(rg, n_tiles);
        XPR_LAUNCH_CHECK("fix_empty_ranges_kernel");
    } else {
        // nothing to sort by (a single tile): one pass over the keys finds the bounds
        const int64_t nthreads = (n + kRangeItems - 1) / kRangeItems;
        tile_ranges_kernel<K><<<(unsigned)((nthreads + 255) / 256), 256, 0, st>>>(
            keys_in, n, (uint32_t)n_tiles, rg, is_aligned16(keys_in));
        XPR_LAUNCH_CHECK("tile_ranges_kernel");
    }
    return XPR_OK;
}

// key = UINT32_MAX - list length: ascending keys = descending lengths (ties keep tile order)
__global__ void worklist_keys_kernel(const int2 *__restrict__ ranges, int n_tiles, uint32_t *__restrict__ keys,
                                     uint32_t *__restrict__ vals) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n_tiles) return;
    const int2 r = ranges[t];
    keys[t] = 0xffffffffu - (uint32_t)(r.y - r.x);
    vals[t] = (uint32_t)t;
}

}  // namespace

size_t worklist_workspace_bytes(int32_t n_tiles) {
    const size_t a = align256((size_t)n_tiles * 4);
    return 3 * a + 256 + workspace_bytes<uint32_t>(n_tiles);
}

int launch_tile_worklist(const int32_t *ranges, int32_t n_tiles, int32_t *worklist, void *ws, size_t ws_bytes,
                         cudaStream_t st) {
    if (n_tiles <= 0) return XPR_OK;
    if (ws_bytes < worklist_workspace_bytes(n_tiles))
        return fail(XPR_ERR_INVALID, "xpr_tile_worklist: workspace %zu < %zu bytes", ws_bytes,
                    worklist_workspace_bytes(n_tiles));
    const size_t a = align256((size_t)n_tiles * 4);
    char *p = reinterpret_cast<char *>(ws);
    uint32_t *keys = reinterpret_cast<uint32_t *>(p);
    uint32_t *keys_sorted = reinterpret_cast<uint32_t *>(p + a);
    uint32_t *vals = reinterpret_cast<uint32_t *>(p + 2 * a);
    int32_t *dummy_ranges = reinterpret_cast<int32_t *>(p + 3 * a);
    worklist_keys_kernel<<<(unsigned)((n_tiles + 255) / 256), 256, 0, st>>>(reinterpret_cast<const int2 *>(ranges),
                                                                            n_tiles, keys, vals);
    XPR_LAUNCH_CHECK("worklist_keys_kernel");
    return radix_sort<uint32_t>(keys, vals, n_tiles, 1, 0, 32, keys_sorted, reinterpret_cast<uint32_t *>(worklist),
                                dummy_ranges, p + 3 * a + 256, workspace_bytes<uint32_t>(n_tiles), st);
}

size_t sort_workspace_bytes(int64_t n, int32_t n_tiles) {
    (void)n_tiles;
    return workspace_bytes<uint64_t>(n);
}

size_t sort_tiles_workspace_bytes(int64_t n, int32_t n_tiles) {
    (void)n_tiles;
    return workspace_bytes<uint32_t>(n);
}

int launch_sort(const uint64_t *keys_in, const uint32_t *vals_in, int64_t n, int32_t n_tiles, int begin_bit,
                uint64_t *keys_out, uint32_t *vals_out, int32_t *ranges, void *ws, size_t ws_bytes, cudaStream_t st) {
    const int end_bit = 32 + bits_for((int64_t)n_tiles - 1);
    return radix_sort<uint64_t>(keys_in, vals_in, n, n_tiles, begin_bit, end_bit, keys_out, vals_out, ranges, ws,
                                ws_bytes, st);
}

int launch_sort_tiles(const uint32_t *tiles_in, const uint32_t *vals_in, int64_t n, int32_t n_tiles,
                      uint32_t *tiles_out, uint32_t *vals_out, int32_t *ranges, void *ws, size_t ws_bytes,
                      cudaStream_t st) {
    return radix_sort<uint32_t>(tiles_in, vals_in, n, n_tiles, 0, bits_for((int64_t)n_tiles - 1), tiles_out,
                                vals_out, ranges, ws, ws_bytes, st);
}

}  // namespace xpr
