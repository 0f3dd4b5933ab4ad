// Rasterizer, second half (Sec. 4.2 "Sort and identify bounds"): stable LSD radix sort of the
// intersection pairs by tile (and depth), then the per-tile segment bounds [start, end).
//
// Keys are either u64 (tile << 32 | depth bits; xpr_sort) or u32 tile ids (xpr_sort_tiles, for
// pairs emitted in depth order, where a stable sort by tile alone gives the (tile, depth) order).
// Each 8-bit pass ranks blocks of keys stably (4096 keys, 16 per thread, in the chained scan; 3072,
// 12 per thread, in reduce-then-scan; warp w owns a contiguous run of 32 x keys-per-thread visited
// in index order; lanes with equal digits are found with one ballot per digit bit), places
// every key at its rank in a block-local sorted copy in shared memory, and writes the copy out in
// order, so consecutive threads write consecutive addresses of one digit's run.  The global start
// of each (block, digit) run comes from one of two schemes:
//   * chained scan (up to kChainedMaxKeys keys, where a sort is short and launch-bound): one
//     histogram kernel counts the digits of every pass in one read of the keys; each pass's
//     scatter block takes its index from a counter (blocks start in index order), publishes its
//     per-digit counts and sums the counts of the blocks before it by looking back through their
//     published words until it meets a block whose running total is known.  Every look-back wait
//     is bounded: a block that polls too long records the timeout in a device flag (read by
//     xpr_device_check) and carries on, and every write is bounds-checked.
//   * reduce-then-scan (larger sorts, where the look-back's latency would lengthen every block's
//     life): per pass, a histogram kernel counts each block's digits into a block-major (block x
//     digit) matrix, and a column scan of it (32-row segment sums, a scan over segments per
//     digit, then the in-place prefix) turns every entry into the run's global offset.
#include "xpr_internal.cuh"

namespace xpr {
namespace {

constexpr int kThreads = 256;
#ifndef XPR_CHAINED_ITEMS
#define XPR_CHAINED_ITEMS 16
#endif
constexpr int kItems = XPR_CHAINED_ITEMS;  // keys per thread of the chained-scan kernels
constexpr int kWarps = kThreads / 32;
constexpr int kWarpKeys = 32 * kItems;    // 512
constexpr int kTile = kThreads * kItems;  // 4096
// Reduce-then-scan kernels: 12 keys per thread, so that the scatter fits 64 registers (4 blocks of
// 256 threads per SM instead of 3 at 16 keys and 80 registers; 0.69 -> 0.64 ms on 48M pairs).
constexpr int kItemsR = 12;
constexpr int kWarpKeysR = 32 * kItemsR;  // 384
constexpr int kTileR = kThreads * kItemsR;  // 3072
constexpr int kRadix = 256;
constexpr int kMaxPasses = 8;             // 64-bit keys
constexpr int kRangeItems = 8;            // keys per thread of the segment-bound kernel
constexpr int kSegRows = 32;              // matrix rows per segment of the column scan
constexpr int64_t kChainedMaxKeys = 1 << 22;  // measured crossover of the two schemes

// Word of (block, digit) in a pass's chained scan: 0 = not yet published; 1 .. kTile + 1 = the
// block's own count of the digit plus one; kPrefixFlag | c = the count c of the digit in this
// block and all blocks before it (c < 2^31 as n < 2^31).
constexpr uint32_t kPrefixFlag = 0x80000000u;
constexpr int kWaitPolls = 1 << 20;       // with the 64 ns back-off, at least ~70 ms per word
constexpr int kLook = 16;                 // earlier blocks' words read at once by the look-back

// Device error bits: 1 = a look-back wait gave up, 2 = a published word was inconsistent or a
// computed position fell outside the output.
__device__ unsigned int g_sort_errors;

__device__ __forceinline__ uint32_t ld_relaxed(const uint32_t *p) {
    uint32_t v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_relaxed(uint32_t *p, uint32_t v) {
    asm volatile("st.relaxed.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

template <typename K>
constexpr size_t chained_smem() {
    return (size_t)kTile * sizeof(K) + (size_t)kTile * 4 + (size_t)kWarps * kRadix * 4 + 3 * (size_t)kRadix * 4 + 64;
}
template <typename K>
constexpr size_t scatter_smem() {
    return (size_t)kTileR * sizeof(K) + (size_t)kTileR * 4 + (size_t)kWarps * kRadix * 4 + 2 * (size_t)kRadix * 4 + 64;
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

// ghist[p][d] += number of keys whose digit in pass p (bits [begin + 8p, min(begin + 8p + 8, end)))
// is d, for all passes in one read of the keys (grid-stride over blocks of kTile keys); the grid
// also zeroes the first pass's chained-scan words.  vec: kin is 16-byte aligned.
template <typename K>
__global__ void __launch_bounds__(kThreads) sort_hist_kernel(const K *__restrict__ kin, int64_t n, int begin_bit,
                                                             int end_bit, int passes, uint32_t *__restrict__ ghist,
                                                             uint4 *__restrict__ status0, int64_t status_vecs,
                                                             bool vec) {
    grid_dep_wait();
    __shared__ uint32_t s[kMaxPasses][kRadix];
    for (int d = threadIdx.x; d < kMaxPasses * kRadix; d += kThreads) (&s[0][0])[d] = 0;
    const int64_t gt = (int64_t)blockIdx.x * kThreads + threadIdx.x, gs = (int64_t)gridDim.x * kThreads;
    for (int64_t i = gt; i < status_vecs; i += gs) status0[i] = make_uint4(0, 0, 0, 0);
    __syncthreads();
    const int64_t nb = (n + kTile - 1) / kTile;
    for (int64_t blk = blockIdx.x; blk < nb; blk += gridDim.x) {
        const int64_t base = blk * kTile + (int64_t)threadIdx.x * kItems;
        K k[kItems];
        const bool full = base + kItems <= n;
        if (vec && full) {
#pragma unroll
            for (int q = 0; q < kItems; q += 4) {
                K v[4];
                load4(kin, base + q, v);
#pragma unroll
                for (int r = 0; r < 4; ++r) k[q + r] = v[r];
            }
        } else {
#pragma unroll
            for (int q = 0; q < kItems; ++q) k[q] = base + q < n ? kin[base + q] : K(0);
        }
        const int m = full ? kItems : (int)max((int64_t)0, n - base);
        for (int p = 0; p < passes; ++p) {
            const int shift = begin_bit + 8 * p;
            const uint32_t mask = (1u << min(8, end_bit - shift)) - 1u;
            // equal neighbouring digits are added as one run
            int prev = -1, run = 0;
#pragma unroll
            for (int q = 0; q < kItems; ++q) {
                if (q < m) {
                    const int d = (int)((uint32_t)(k[q] >> shift) & mask);
                    if (d == prev) {
                        ++run;
                    } else {
                        if (run) atomicAdd(&s[p][prev], (uint32_t)run);
                        prev = d;
                        run = 1;
                    }
                }
            }
            if (run) atomicAdd(&s[p][prev], (uint32_t)run);
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < passes * kRadix; i += kThreads) {
        const uint32_t c = (&s[0][0])[i];
        if (c) atomicAdd(&ghist[i], c);
    }
}


// Reduce-then-scan, per pass: hist[b][d] = number of keys of block b with digit d.  vec: kin is 16-byte aligned.
template <typename K>
__global__ void __launch_bounds__(kThreads) radix_hist_kernel(const K *__restrict__ kin, int64_t n, int shift,
                                                              uint32_t mask, int32_t *__restrict__ hist, bool vec) {
    grid_dep_wait();
    __shared__ int s[kWarps][kRadix];
    for (int d = threadIdx.x; d < kWarps * kRadix; d += kThreads) (&s[0][0])[d] = 0;
    __syncthreads();
    const int w = threadIdx.x >> 5;
    const int64_t base = (int64_t)blockIdx.x * kTileR + (int64_t)threadIdx.x * kItemsR;
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
    if (vec && base + kItemsR <= n) {
#pragma unroll
        for (int q = 0; q < kItemsR; q += 4) {
            K k[4];
            load4(kin, base + q, k);
#pragma unroll
            for (int r = 0; r < 4; ++r) add(k[r]);
        }
    } else {
        for (int q = 0; q < kItemsR; ++q)
            if (base + q < n) add(kin[base + q]);
    }
    if (run) atomicAdd(&s[w][prev], run);
    __syncthreads();
    int sum = 0;
#pragma unroll
    for (int ww = 0; ww < kWarps; ++ww) sum += s[ww][threadIdx.x];
    hist[(int64_t)blockIdx.x * kRadix + threadIdx.x] = sum;
}

// Column scan of the (block x digit) matrix, step 1: part[g][d] = sum of rows [32 g, 32 g + 32).
__global__ void __launch_bounds__(kRadix) colsum_kernel(const int32_t *__restrict__ hist, int64_t nb,
                                                        int32_t *__restrict__ part) {
    grid_dep_wait();
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
    grid_dep_wait();
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
    grid_dep_wait();
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


// The count of digit d0 in all blocks before block b > 0 of a chained-scan pass: a word not yet
// published is polled alone; after each step over published counts the window of words read at
// once grows (1, 4, 16), so that one round trip walks up to kLook blocks.  A word still unpublished
// after max_polls polls sets the timeout flag and ends the walk (the count is then short); walking
// past block 0, which always publishes its running total, sets the consistency flag.
__device__ __forceinline__ uint32_t lookback(const uint32_t *status, int b, int d0, int max_polls) {
    uint32_t excl = 0;
    int j = b - 1, polls = 0, win = 1;
    for (;;) {
        uint32_t wv[kLook];
#pragma unroll
        for (int q = 0; q < kLook; ++q)
            wv[q] = (q < win && j - q >= 0) ? ld_relaxed(status + (size_t)(j - q) * kRadix + d0) : 0u;
        int adv = 0;
        bool stop = false, found = false;
#pragma unroll
        for (int q = 0; q < kLook; ++q) {
            if (!stop) {
                const uint32_t sw = wv[q];
                if (sw == 0u) {
                    stop = true;  // not yet published (or outside the window)
                } else if (sw & kPrefixFlag) {
                    excl += sw & ~kPrefixFlag;
                    stop = found = true;
                } else {
                    excl += sw - 1u;
                    ++adv;
                }
            }
        }
        if (found) return excl;
        j -= adv;
        if (j < 0) {
            atomicOr(&g_sort_errors, 2u);
            return excl;
        }
        if (adv == 0) {
            if (++polls >= max_polls) {
                atomicOr(&g_sort_errors, 1u);
                return excl;
            }
            __nanosleep(64);
            win = 1;
        } else {
            polls = 0;
            win = min(4 * win, kLook);
        }
    }
}

// Self-test of the bounded wait: every thread looks back from block 1 at block 0's words, which
// the caller has zeroed and nothing publishes, so each wait runs out after max_polls polls.
__global__ void lookback_selftest_kernel(const uint32_t *status, int max_polls, uint32_t *out) {
    out[threadIdx.x] = lookback(status, 1, (int)threadIdx.x, max_polls);
}

// Exclusive scan over the block's 256 threads of two ints at once (one per digit); totals unused.
__device__ __forceinline__ void digit_scan2(int a, int b, int &ea, int &eb, int2 *s_wsum) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int x = a, y = b;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int u = __shfl_up_sync(0xffffffffu, x, o), v = __shfl_up_sync(0xffffffffu, y, o);
        if (lane >= o) {
            x += u;
            y += v;
        }
    }
    if (lane == 31) s_wsum[w] = make_int2(x, y);
    __syncthreads();
    int pa = 0, pb = 0;
    for (int ww = 0; ww < w; ++ww) {
        pa += s_wsum[ww].x;
        pb += s_wsum[ww].y;
    }
    ea = pa + x - a;
    eb = pb + y - b;
}

// Chained-scan scatter of one pass over bits [shift, shift + NB) (NB <= 8).  status: this pass's
// words (nb x 256); status_next: the next pass's, whose row of this block is zeroed here (NULL on
// the last pass); ghist: this pass's global digit counts; ctr: this pass's block counter (from 0).
// Last pass only (ranges non-NULL): the output is in final order, and inside a block's local run
// the keys of one tile are contiguous (one digit group, ordered by the lower digits), so the
// first and last key of each local tile run give that tile's segment bounds through one atomic
// min / max each (ranges start as [INT_MAX, 0) and untouched tiles are reset to [0, 0) after).
// kout NULL: the sorted keys are not written (only their segment bounds are wanted).
template <typename K, int NB>
__global__ void __launch_bounds__(kThreads)
    chained_scatter_kernel(const K *__restrict__ kin, const uint32_t *__restrict__ vin, K *__restrict__ kout,
                           uint32_t *__restrict__ vout, int64_t n, int shift, const uint32_t *__restrict__ ghist,
                           uint32_t *status, uint32_t *__restrict__ status_next, uint32_t *ctr,
                           int2 *__restrict__ ranges, uint32_t n_tiles) {
    grid_dep_wait();
    constexpr uint32_t kMask = (1u << NB) - 1u;
    extern __shared__ __align__(16) unsigned char smem[];
    K *s_key = reinterpret_cast<K *>(smem);
    uint32_t *s_val = reinterpret_cast<uint32_t *>(smem + (size_t)kTile * sizeof(K));
    int(*s_hist)[kRadix] = reinterpret_cast<int(*)[kRadix]>(smem + (size_t)kTile * (sizeof(K) + 4));
    int *s_start = reinterpret_cast<int *>(smem + (size_t)kTile * (sizeof(K) + 4) + (size_t)kWarps * kRadix * 4);
    int64_t *s_gofs = reinterpret_cast<int64_t *>(s_start + kRadix);  // kRadix int64 after s_start
    __shared__ int2 s_wsum[kWarps];
    __shared__ int s_bid;

    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (threadIdx.x == 0) s_bid = (int)atomicAdd(ctr, 1u);
    for (int d = threadIdx.x; d < kWarps * kRadix; d += kThreads) (&s_hist[0][0])[d] = 0;
    __syncthreads();
    const int b = s_bid;
    if (status_next) status_next[(size_t)b * kRadix + threadIdx.x] = 0u;
    const int64_t block_base = (int64_t)b * kTile;
    const K *kb = kin + block_base;
    const uint32_t *vb = vin + block_base;
    const int count = (int)min((int64_t)kTile, n - block_base);
    const int wbase = w * kWarpKeys;
    const unsigned lt_mask = (1u << lane) - 1u;
    // all of the thread's keys (and, for 4-byte keys, values) are loaded before any ranking so
    // that a warp has kItems loads in flight instead of one per round
    constexpr bool kHoldVals = sizeof(K) <= 4;
    K kreg[kItems];
    uint32_t vreg[kHoldVals ? kItems : 1];
#pragma unroll
    for (int r = 0; r < kItems; ++r) {
        const int idx = wbase + r * 32 + lane;
        kreg[r] = idx < count ? kb[idx] : K(0);
        if (kHoldVals) vreg[kHoldVals ? r : 0] = idx < count ? vb[idx] : 0u;
    }
    // Lanes with equal digits: one ballot per digit bit; the group's lowest lane alone reads and
    // bumps the warp's running count of the digit and hands the old count to its group.
    int dr[kItems];
#pragma unroll
    for (int r = 0; r < kItems; ++r) {
        const int idx = wbase + r * 32 + lane;
        const bool valid = idx < count;
        const uint32_t d = valid ? (uint32_t)(kreg[r] >> shift) & kMask : 0u;
        unsigned peers = __ballot_sync(0xffffffffu, valid);
#pragma unroll
        for (int bit = 0; bit < NB; ++bit) {
            const unsigned bal = __ballot_sync(0xffffffffu, (d >> bit) & 1u);
            peers &= ~(bal ^ (0u - ((d >> bit) & 1u)));
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
    // publish this block's count of the digit (block 0: its running total) at once
    uint32_t *my = status + (size_t)b * kRadix + d0;
    st_relaxed(my, b == 0 ? (kPrefixFlag | (uint32_t)tot) : (uint32_t)tot + 1u);
    // start of the digit in the local order and in the pass's output
    int start, gstart;
    digit_scan2(tot, (int)ghist[d0], start, gstart, s_wsum);
    s_start[d0] = start;
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
    // look back (after the placement, so that the blocks before this one have had time to publish)
    uint32_t excl = 0;
    if (b > 0) {
        excl = lookback(status, b, d0, kWaitPolls);
        st_relaxed(my, kPrefixFlag | (excl + (uint32_t)tot));
    }
    s_gofs[d0] = (int64_t)gstart + excl - start;
    __syncthreads();
    // write the block's sorted run: consecutive threads, consecutive output addresses within a digit
    bool bad = false;
    for (int s = threadIdx.x; s < count; s += kThreads) {
        const K k = s_key[s];
        const int d = (int)((uint32_t)(k >> shift) & kMask);
        const int64_t g = s_gofs[d] + s;
        if ((uint64_t)g >= (uint64_t)n) {
            bad = true;
            continue;
        }
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
    if (bad) atomicOr(&g_sort_errors, 2u);
}

// Reduce-then-scan scatter of one pass; offs[b][d] = global output offset of block b's run of
// digit d.  Last pass only (ranges non-NULL): the output is in final order, and inside a block's local run
// the keys of one tile are contiguous (one digit group, ordered by the lower digits), so the
// first and last key of each local tile run give that tile's segment bounds through one atomic
// min / max each (ranges start as [INT_MAX, 0) and untouched tiles are reset to [0, 0) after).
// kout NULL: the sorted keys are not written (only their segment bounds are wanted).
template <typename K>
__global__ void __launch_bounds__(kThreads, 4) radix_scatter_kernel(const K *__restrict__ kin,
                                                                 const uint32_t *__restrict__ vin,
                                                                 K *__restrict__ kout, uint32_t *__restrict__ vout,
                                                                 int64_t n, int shift, uint32_t mask,
                                                                 const int32_t *__restrict__ offs,
                                                                 int2 *__restrict__ ranges, uint32_t n_tiles) {
    grid_dep_wait();
    extern __shared__ __align__(16) unsigned char smem[];
    K *s_key = reinterpret_cast<K *>(smem);
    uint32_t *s_val = reinterpret_cast<uint32_t *>(smem + (size_t)kTileR * sizeof(K));
    int(*s_hist)[kRadix] = reinterpret_cast<int(*)[kRadix]>(smem + (size_t)kTileR * (sizeof(K) + 4));
    int *s_start = reinterpret_cast<int *>(smem + (size_t)kTileR * (sizeof(K) + 4) + (size_t)kWarps * kRadix * 4);
    int *s_gofs = s_start + kRadix;
    int *s_wsum = s_gofs + kRadix;  // kWarps partial sums for the digit scan

    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int d = threadIdx.x; d < kWarps * kRadix; d += kThreads) (&s_hist[0][0])[d] = 0;
    __syncthreads();
    const int64_t block_base = (int64_t)blockIdx.x * kTileR;
    const K *kb = kin + block_base;
    const uint32_t *vb = vin + block_base;
    const int count = (int)min((int64_t)kTileR, n - block_base);
    const int wbase = w * kWarpKeysR;
    const unsigned lt_mask = (1u << lane) - 1u;
    // Lanes with equal digits are found with one ballot per digit bit (the match instruction runs
    // on a narrow pipe that limited this kernel); the group's lowest lane alone reads and bumps
    // the warp's running count of the digit and hands the old count to its group by a shuffle.
    const int nbits = __popc(mask);
    // all of the thread's keys (and, for 4-byte keys, values) are loaded before any ranking so
    // that a warp has kItemsR loads in flight instead of one per round
    constexpr bool kHoldVals = sizeof(K) <= 4;
    K kreg[kItemsR];
    uint32_t vreg[kHoldVals ? kItemsR : 1];
#pragma unroll
    for (int r = 0; r < kItemsR; ++r) {
        const int idx = wbase + r * 32 + lane;
        kreg[r] = idx < count ? kb[idx] : K(0);
        if (kHoldVals) vreg[kHoldVals ? r : 0] = idx < count ? vb[idx] : 0u;
    }
    int dr[kItemsR];
#pragma unroll
    for (int r = 0; r < kItemsR; ++r) {
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
    for (int r = 0; r < kItemsR; ++r) {
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
    grid_dep_wait();
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n_tiles) ranges[t] = make_int2(0x7fffffff, 0);
}

__global__ void fix_empty_ranges_kernel(int2 *__restrict__ ranges, int n_tiles) {
    grid_dep_wait();
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

// Workspace: the ping-pong copies of keys and values (only for more than one pass: a single pass
// reads the input and writes the output), two (block x digit) matrices (chained: the words of the
// current and the next pass; reduce-then-scan: the offset matrix and the segment sums) and the
// digit counts with the block counters (reduce-then-scan: the digit totals).
template <typename K>
size_t workspace_bytes(int64_t n, int passes = kMaxPasses) {
    const int64_t tk = kTileR < kTile ? kTileR : kTile;  // the smaller tile: the larger block count
    const int64_t nb = max((int64_t)1, (n + tk - 1) / tk);
    const size_t alt = passes > 1 ? align256((size_t)n * sizeof(K)) + align256((size_t)n * 4) : 0;
    return alt + 2 * align256((size_t)nb * kRadix * 4) + align256((size_t)kMaxPasses * (kRadix + 1) * 4);
}

template <typename K, int NB>
int launch_chained(int64_t nb, cudaStream_t st, const K *kin, const uint32_t *vin, K *kout, uint32_t *vout, int64_t n,
                   int shift, const uint32_t *ghist, uint32_t *status, uint32_t *status_next, uint32_t *ctr,
                   int2 *ranges, uint32_t n_tiles) {
    // the dynamic shared-memory limit is a per-function attribute of the current device's module
    // (one value per instantiation, so concurrent callers all set the same limit)
    XPR_CUDA_TRY(cudaFuncSetAttribute(chained_scatter_kernel<K, NB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)chained_smem<K>()));
    XPR_CUDA_TRY(launch_dependent(chained_scatter_kernel<K, NB>, dim3((unsigned)nb), dim3(kThreads), chained_smem<K>(),
                                  st, kin, vin, kout, vout, n, shift, ghist, status, status_next, ctr, ranges, n_tiles));
    XPR_LAUNCH_CHECK("chained_scatter_kernel");
    return XPR_OK;
}

// The pass's digit width is a template argument so that the ballot loop unrolls.
template <typename K, typename... A>
int launch_chained_bits(int nbits, A... a) {
    switch (nbits) {
        case 1: return launch_chained<K, 1>(a...);
        case 2: return launch_chained<K, 2>(a...);
        case 3: return launch_chained<K, 3>(a...);
        case 4: return launch_chained<K, 4>(a...);
        case 5: return launch_chained<K, 5>(a...);
        case 6: return launch_chained<K, 6>(a...);
        case 7: return launch_chained<K, 7>(a...);
        default: return launch_chained<K, 8>(a...);
    }
}

// Sorts (kin, vin) by key bits [begin_bit, end_bit) into (kout, vout), then finds tile ranges
// (ranges NULL: none are wanted).
template <typename K>
int radix_sort(const K *keys_in, const uint32_t *vals_in, int64_t n, int32_t n_tiles, int begin_bit, int end_bit,
               K *keys_out, uint32_t *vals_out, int32_t *ranges, void *ws, size_t ws_bytes, cudaStream_t st) {
    if (ranges) XPR_CUDA_TRY(cudaMemsetAsync(ranges, 0, (size_t)n_tiles * 2 * sizeof(int32_t), st));
    if (n == 0) return XPR_OK;
    if (n > 0x7fffffffLL) return fail(XPR_ERR_INVALID, "sort: more than 2^31 - 1 keys");
    const int passes = begin_bit < end_bit ? (end_bit - begin_bit + 7) / 8 : 0;
    if (passes > kMaxPasses) return fail(XPR_ERR_INVALID, "sort: %d passes > %d", passes, kMaxPasses);
    if (ws_bytes < workspace_bytes<K>(n, passes))
        return fail(XPR_ERR_INVALID, "sort: workspace %zu bytes < required %zu", ws_bytes,
                    workspace_bytes<K>(n, passes));
    const bool chained = n <= kChainedMaxKeys;
    const int tile_keys = chained ? kTile : kTileR;
    const int64_t nb = (n + tile_keys - 1) / tile_keys;
    const int64_t nseg = (nb + kSegRows - 1) / kSegRows;
    char *p = reinterpret_cast<char *>(ws);
    K *alt_k = reinterpret_cast<K *>(p);  // the ping-pong copies: used (and present) for 2+ passes only
    if (passes > 1) p += align256((size_t)n * sizeof(K));
    uint32_t *alt_v = reinterpret_cast<uint32_t *>(p);
    if (passes > 1) p += align256((size_t)n * 4);
    uint32_t *mat[2];
    mat[0] = reinterpret_cast<uint32_t *>(p);
    p += align256((size_t)nb * kRadix * 4);
    mat[1] = reinterpret_cast<uint32_t *>(p);
    p += align256((size_t)nb * kRadix * 4);
    uint32_t *ghist = reinterpret_cast<uint32_t *>(p);  // kMaxPasses x kRadix counts, then kMaxPasses counters
    uint32_t *ctr = ghist + kMaxPasses * kRadix;

    int2 *rg = reinterpret_cast<int2 *>(ranges);
    if (passes == 0) {
        if (keys_out)
            XPR_CUDA_TRY(cudaMemcpyAsync(keys_out, keys_in, (size_t)n * sizeof(K), cudaMemcpyDeviceToDevice, st));
        XPR_CUDA_TRY(cudaMemcpyAsync(vals_out, vals_in, (size_t)n * 4, cudaMemcpyDeviceToDevice, st));
        // nothing to sort by (a single tile): one pass over the keys finds the bounds
        if (!rg) return XPR_OK;
        const int64_t nthreads = (n + kRangeItems - 1) / kRangeItems;
        tile_ranges_kernel<K><<<(unsigned)((nthreads + 255) / 256), 256, 0, st>>>(
            keys_in, n, (uint32_t)n_tiles, rg, is_aligned16(keys_in));
        XPR_LAUNCH_CHECK("tile_ranges_kernel");
        return XPR_OK;
    }
    const unsigned tgrid = (unsigned)((n_tiles + 255) / 256);
    if (rg) {
        XPR_CUDA_TRY(launch_dependent(init_ranges_kernel, dim3(tgrid), dim3(256), 0, st, rg, (int)n_tiles));
        XPR_LAUNCH_CHECK("init_ranges_kernel");
    }
    if (chained) {
        int dev = 0, sms = 0;
        XPR_CUDA_TRY(cudaGetDevice(&dev));
        XPR_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        XPR_CUDA_TRY(cudaMemsetAsync(ghist, 0, (size_t)kMaxPasses * (kRadix + 1) * 4, st));
        const unsigned hgrid = (unsigned)min(nb, (int64_t)8 * max(sms, 1));
        XPR_CUDA_TRY(launch_dependent(sort_hist_kernel<K>, dim3(hgrid), dim3(kThreads), 0, st, keys_in, n, begin_bit,
                                      end_bit, passes, ghist, reinterpret_cast<uint4 *>(mat[0]), nb * kRadix / 4,
                                      is_aligned16(keys_in)));
        XPR_LAUNCH_CHECK("sort_hist_kernel");
    }
    const K *src_k = keys_in;
    const uint32_t *src_v = vals_in;
    for (int pass = 0; pass < passes; ++pass) {
        const int shift = begin_bit + 8 * pass;
        const int nbits = min(8, end_bit - shift);
        const bool to_out = ((passes - 1 - pass) % 2) == 0;
        const bool last = pass == passes - 1;
        uint32_t *dst_v = to_out ? vals_out : alt_v;
        // keys: keys_out / alt ping-pong; without keys_out the last pass writes no keys and the
        // others alternate alt, keys_in (the caller's input doubles as the second buffer)
        K *dst_k = keys_out ? (to_out ? keys_out : alt_k)
                            : (last ? nullptr : ((pass % 2) == 0 ? alt_k : const_cast<K *>(keys_in)));
        int s;
        if (chained) {
            s = launch_chained_bits<K>(nbits, nb, st, src_k, src_v, dst_k, dst_v, n, shift,
                                       (const uint32_t *)(ghist + pass * kRadix), mat[pass % 2],
                                       last ? (uint32_t *)nullptr : mat[(pass + 1) % 2], ctr + pass,
                                       last ? rg : (int2 *)nullptr, (uint32_t)n_tiles);
        } else {
            int32_t *hist = reinterpret_cast<int32_t *>(mat[0]);
            int32_t *part = reinterpret_cast<int32_t *>(mat[1]);
            int32_t *dtot = reinterpret_cast<int32_t *>(ghist);
            const uint32_t mask = (1u << nbits) - 1u;
            XPR_CUDA_TRY(launch_dependent(radix_hist_kernel<K>, dim3((unsigned)nb), dim3(kThreads), 0, st, src_k, n,
                                          shift, mask, hist, is_aligned16(src_k)));
            XPR_LAUNCH_CHECK("radix_hist_kernel");
            XPR_CUDA_TRY(launch_dependent(colsum_kernel, dim3((unsigned)nseg), dim3(kRadix), 0, st,
                                          (const int32_t *)hist, nb, part));
            XPR_LAUNCH_CHECK("colsum_kernel");
            XPR_CUDA_TRY(launch_dependent(segscan_kernel, dim3(kRadix), dim3(1024), 0, st, part, nseg, dtot));
            XPR_LAUNCH_CHECK("segscan_kernel");
            XPR_CUDA_TRY(launch_dependent(colapply_kernel, dim3((unsigned)nseg), dim3(kRadix), 0, st, hist, nb,
                                          (const int32_t *)part, (const int32_t *)dtot));
            XPR_LAUNCH_CHECK("colapply_kernel");
            XPR_CUDA_TRY(cudaFuncSetAttribute(radix_scatter_kernel<K>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                              (int)scatter_smem<K>()));
            XPR_CUDA_TRY(launch_dependent(radix_scatter_kernel<K>, dim3((unsigned)nb), dim3(kThreads),
                                          scatter_smem<K>(), st, src_k, src_v, dst_k, dst_v, n, shift, mask,
                                          (const int32_t *)hist, last ? rg : (int2 *)nullptr, (uint32_t)n_tiles));
            XPR_LAUNCH_CHECK("radix_scatter_kernel");
            s = XPR_OK;
        }
        if (s != XPR_OK) return s;
        src_k = dst_k;
        src_v = dst_v;
    }
    if (rg) {
        XPR_CUDA_TRY(launch_dependent(fix_empty_ranges_kernel, dim3(tgrid), dim3(256), 0, st, rg, (int)n_tiles));
        XPR_LAUNCH_CHECK("fix_empty_ranges_kernel");
    }
    return XPR_OK;
}

// key = UINT32_MAX - list length: ascending keys = descending lengths (ties keep tile order)
__global__ void worklist_keys_kernel(const int2 *__restrict__ ranges, int n_tiles, uint32_t *__restrict__ keys,
                                     uint32_t *__restrict__ vals) {
    grid_dep_wait();
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n_tiles) return;
    const int2 r = ranges[t];
    keys[t] = 0xffffffffu - (uint32_t)(r.y - r.x);
    vals[t] = (uint32_t)t;
}

}  // namespace

int lookback_selftest(uint32_t *zeroed, int max_polls, cudaStream_t st) {
    lookback_selftest_kernel<<<1, kRadix, 0, st>>>(zeroed, max_polls, zeroed + kRadix);
    XPR_LAUNCH_CHECK("lookback_selftest_kernel");
    return XPR_OK;
}

int sort_device_errors(unsigned *bits) {
    unsigned v = 0;
    XPR_CUDA_TRY(cudaDeviceSynchronize());
    XPR_CUDA_TRY(cudaMemcpyFromSymbol(&v, g_sort_errors, sizeof(v)));
    if (v) {
        const unsigned zero = 0;
        XPR_CUDA_TRY(cudaMemcpyToSymbol(g_sort_errors, &zero, sizeof(zero)));
    }
    *bits = v;
    return XPR_OK;
}

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
    XPR_CUDA_TRY(launch_dependent(worklist_keys_kernel, dim3((unsigned)((n_tiles + 255) / 256)), dim3(256), 0, st,
                                  reinterpret_cast<const int2 *>(ranges), n_tiles, keys, vals));
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

int launch_sort_u32_bits(const uint32_t *keys_in, const uint32_t *vals_in, int64_t n, int32_t n_tiles, int begin_bit,
                         int end_bit, uint32_t *keys_out, uint32_t *vals_out, int32_t *ranges, void *ws,
                         size_t ws_bytes, cudaStream_t st) {
    return radix_sort<uint32_t>(keys_in, vals_in, n, n_tiles, begin_bit, end_bit, keys_out, vals_out, ranges, ws,
                                ws_bytes, st);
}

}  // namespace xpr
