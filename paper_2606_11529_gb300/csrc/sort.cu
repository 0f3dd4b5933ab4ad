// Rasterizer, second half (Sec. 4.2 "Sort and identify bounds"): stable LSD radix sort of the
// intersection pairs by tile (and depth), then the per-tile segment bounds [start, end).
//
// Keys are either u64 (tile << 32 | depth bits; xpr_sort) or u32 tile ids (xpr_sort_tiles, for
// pairs emitted in depth order, where a stable sort by tile alone gives the (tile, depth) order).
// Each 8-bit pass is reduce-then-scan: a histogram kernel writes per-block digit counts in
// digit-major order, the device-wide exclusive scan turns them into global output offsets, and
// the scatter kernel
//   1. ranks its keys stably: warp w owns a contiguous run of 256 keys visited in index order,
//      __match_any_sync groups equal digits within each round of 32;
//   2. places every key at its rank in a block-local sorted copy in shared memory;
//   3. writes the local copy out in order, so the threads of a warp write consecutive addresses
//      of one digit's output run (coalesced) instead of 32 scattered buckets.
#include "xpr_internal.cuh"

namespace xpr {
namespace {

constexpr int kThreads = 256;
constexpr int kItems = 8;
constexpr int kWarps = kThreads / 32;
constexpr int kWarpKeys = 32 * kItems;   // 256
constexpr int kTile = kThreads * kItems;  // 2048
constexpr int kRadix = 256;

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

template <typename K>
__global__ void __launch_bounds__(kThreads) radix_hist_kernel(const K *__restrict__ kin, int64_t n, int shift,
                                                              uint32_t mask, int32_t *__restrict__ hist,
                                                              int64_t nb) {
    __shared__ int s[kRadix];
    s[threadIdx.x] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * kTile;
#pragma unroll 4
    for (int k = threadIdx.x; k < kTile; k += kThreads) {
        const int64_t j = base + k;
        if (j < n) atomicAdd(&s[(uint32_t)(kin[j] >> shift) & mask], 1);
    }
    __syncthreads();
    hist[(int64_t)threadIdx.x * nb + blockIdx.x] = s[threadIdx.x];
}

template <typename K>
__global__ void __launch_bounds__(kThreads) radix_scatter_kernel(const K *__restrict__ kin,
                                                                 const uint32_t *__restrict__ vin,
                                                                 K *__restrict__ kout, uint32_t *__restrict__ vout,
                                                                 int64_t n, int shift, uint32_t mask,
                                                                 const int32_t *__restrict__ digit_off,
                                                                 int64_t nb) {
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
    const int64_t base = block_base + (int64_t)w * kWarpKeys;
    const int count = (int)min((int64_t)kTile, n - block_base);
    const unsigned lt_mask = (1u << lane) - 1u;
    // only (digit << 16 | rank within the warp) is kept in registers; keys and values are re-read
    // (from L2, just touched) when they are placed
    int dr[kItems];
#pragma unroll
    for (int r = 0; r < kItems; ++r) {
        const int64_t j = base + r * 32 + lane;
        const bool valid = j < n;
        const int d = valid ? (int)((uint32_t)(kin[j] >> shift) & mask) : kRadix;  // kRadix = padding
        const unsigned peers = __match_any_sync(0xffffffffu, d);
        const int leader = __ffs(peers) - 1;
        int cur = 0;
        if (valid) cur = s_hist[w][d];
        __syncwarp();
        if (valid && lane == leader) s_hist[w][d] = cur + __popc(peers);
        __syncwarp();
        dr[r] = (d << 16) | (cur + __popc(peers & lt_mask));
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
    s_gofs[d0] = digit_off[(int64_t)d0 * nb + blockIdx.x] - start;
    __syncthreads();
    // place every key at its local rank
#pragma unroll
    for (int r = 0; r < kItems; ++r) {
        const int64_t j = base + r * 32 + lane;
        if (j < n) {
            const int d = dr[r] >> 16;
            const int pos = s_start[d] + s_hist[w][d] + (dr[r] & 0xffff);
            s_key[pos] = kin[j];
            s_val[pos] = vin[j];
        }
    }
    __syncthreads();
    // write the block's sorted run: consecutive threads, consecutive output addresses within a digit
    for (int s = threadIdx.x; s < count; s += kThreads) {
        const K k = s_key[s];
        const int d = (int)((uint32_t)(k >> shift) & mask);
        const int64_t g = (int64_t)s_gofs[d] + s;
        kout[g] = k;
        vout[g] = s_val[s];
    }
}

template <typename K>
__global__ void tile_ranges_kernel(const K *__restrict__ keys, int64_t n, uint32_t n_tiles,
                                   int2 *__restrict__ ranges) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint32_t t = tile_of<K>(keys[i]);
    if (t >= n_tiles) return;  // keys outside the tile grid have no segment
    if (i == 0 || tile_of<K>(keys[i - 1]) != t) ranges[t].x = (int)i;
    if (i == n - 1 || tile_of<K>(keys[i + 1]) != t) ranges[t].y = (int)(i + 1);
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

template <typename K>
size_t workspace_bytes(int64_t n) {
    const int64_t nb = (n + kTile - 1) / kTile;
    const int64_t nh = (int64_t)kRadix * (nb > 0 ? nb : 1);
    return align256((size_t)n * sizeof(K)) + align256((size_t)n * 4) + align256((size_t)(nh + 1) * 4) +
           scan_partials_bytes(nh);
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
    XPR_CUDA_TRY(cudaFuncSetAttribute(radix_scatter_kernel<K>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)scatter_smem<K>()));
    const int64_t nb = (n + kTile - 1) / kTile;
    const int64_t nh = (int64_t)kRadix * nb;
    char *p = reinterpret_cast<char *>(ws);
    K *alt_k = reinterpret_cast<K *>(p);
    p += align256((size_t)n * sizeof(K));
    uint32_t *alt_v = reinterpret_cast<uint32_t *>(p);
    p += align256((size_t)n * 4);
    int32_t *hist = reinterpret_cast<int32_t *>(p);
    p += align256((size_t)(nh + 1) * 4);
    void *scan_ws = p;

    const int passes = begin_bit < end_bit ? (end_bit - begin_bit + 7) / 8 : 0;
    if (passes == 0) {
        XPR_CUDA_TRY(cudaMemcpyAsync(keys_out, keys_in, (size_t)n * sizeof(K), cudaMemcpyDeviceToDevice, st));
        XPR_CUDA_TRY(cudaMemcpyAsync(vals_out, vals_in, (size_t)n * 4, cudaMemcpyDeviceToDevice, st));
    }
    const K *src_k = keys_in;
    const uint32_t *src_v = vals_in;
    for (int pass = 0; pass < passes; ++pass) {
        const int shift = begin_bit + 8 * pass;
        const int nbits = min(8, end_bit - shift);
        const uint32_t mask = (1u << nbits) - 1u;
        const bool to_out = ((passes - 1 - pass) % 2) == 0;
        K *dst_k = to_out ? keys_out : alt_k;
        uint32_t *dst_v = to_out ? vals_out : alt_v;
        radix_hist_kernel<K><<<(unsigned)nb, kThreads, 0, st>>>(src_k, n, shift, mask, hist, nb);
        XPR_LAUNCH_CHECK("radix_hist_kernel");
        int s = launch_exclusive_scan(hist, hist, nh, scan_ws, nullptr, st);
        if (s != XPR_OK) return s;
        radix_scatter_kernel<K><<<(unsigned)nb, kThreads, scatter_smem<K>(), st>>>(src_k, src_v, dst_k, dst_v, n,
                                                                                   shift, mask, hist, nb);
        XPR_LAUNCH_CHECK("radix_scatter_kernel");
        src_k = dst_k;
        src_v = dst_v;
    }
    tile_ranges_kernel<K><<<(unsigned)((n + 255) / 256), 256, 0, st>>>(keys_out, n, (uint32_t)n_tiles,
                                                                       reinterpret_cast<int2 *>(ranges));
    XPR_LAUNCH_CHECK("tile_ranges_kernel");
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
