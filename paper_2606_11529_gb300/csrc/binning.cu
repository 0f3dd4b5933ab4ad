// Rasterizer, first half (Sec. 4.2): Replicate, Assign tile ID, Cull.
//
// For primitive i and slot r of its half-open tile bounding box (row-major,
// x = xmin + r mod w, y = ymin + r div w, t = y W' + x) the pair is kept iff the StopThePop
// cull of Listing 1 tile_cull passes: the largest response of the Gaussian over the tile is at
// mu_2D when mu_2D lies in the tile, else at the best point of the (at most two) tile edges
// facing mu_2D; on an edge the 1-D quadratic is minimised in closed form and clamped to the edge.
// The decision is taken in FP32 with one correctly rounded IEEE operation per step (explicit
// __f*_rn intrinsics, no contraction), so it is reproducible bit for bit.
//
// Two passes over the primitives (count, then emit at the scanned offsets) give exact
// intersection counts: culled pairs are never written, so the sort moves only survivors.
#include "xpr_internal.cuh"

namespace xpr {
namespace {

__device__ __forceinline__ float quad_half(float c0, float c1, float c2, float dx, float dy) {
    float a = __fmul_rn(__fmul_rn(dx, dx), c0);
    float b = __fmul_rn(__fmul_rn(dx, dy), c1);
    b = __fadd_rn(b, b);
    float c = __fmul_rn(__fmul_rn(dy, dy), c2);
    return __fmul_rn(0.5f, __fadd_rn(__fadd_rn(a, b), c));
}

struct CullData {
    float mx, my, c0, c1, c2, lt;
};

// Tile bounds are inclusive pixel coordinates: x0 = tx w, x1 = min(tx w + w - 1, W - 1).
__device__ __forceinline__ bool tile_keep(const CullData &d, float x0, float y0, float x1, float y1) {
    const bool outx = (d.mx < x0) || (d.mx > x1);
    const bool outy = (d.my < y0) || (d.my > y1);
    if (!outx && !outy) return 0.f <= d.lt;
    float best = __int_as_float(0x7f800000);
    if (outx) {
        const float ex = d.mx < x0 ? x0 : x1;
        const float dx = __fsub_rn(d.mx, ex);
        float ys = __fadd_rn(d.my, __fdiv_rn(__fmul_rn(d.c1, dx), d.c2));
        ys = fminf(fmaxf(ys, y0), y1);
        const float dy = __fsub_rn(d.my, ys);
        best = fminf(best, quad_half(d.c0, d.c1, d.c2, dx, dy));
    }
    if (outy) {
        const float ey = d.my < y0 ? y0 : y1;
        const float dy = __fsub_rn(d.my, ey);
        float xs = __fadd_rn(d.mx, __fdiv_rn(__fmul_rn(d.c1, dy), d.c0));
        xs = fminf(fmaxf(xs, x0), x1);
        const float dx = __fsub_rn(d.mx, xs);
        best = fminf(best, quad_half(d.c0, d.c1, d.c2, dx, dy));
    }
    return best <= d.lt;
}

__device__ __forceinline__ CullData load_cull(const float *__restrict__ rec, int64_t i) {
    const float4 *p = reinterpret_cast<const float4 *>(rec + (size_t)i * XPR_REC_FLOATS);
    float4 a = __ldg(p), b = __ldg(p + 1), c = __ldg(p + 2);
    CullData d;
    d.mx = a.x;
    d.my = a.y;
    d.c0 = a.z;
    d.c1 = a.w;
    d.c2 = b.x;
    d.lt = c.z;
    return d;
}

struct Grid {
    int W, H, tw, th, Wt, Ht;
};

constexpr unsigned kFullMask = 0xffffffffu;
constexpr int kSmallBox = 16;  // boxes with more tiles than this are walked by a whole warp

__device__ __forceinline__ bool keep_tile(const CullData &d, const Grid &g, int tx, int ty) {
    const float x0 = (float)(tx * g.tw), x1 = (float)min(tx * g.tw + g.tw - 1, g.W - 1);
    const float y0 = (float)(ty * g.th), y1 = (float)min(ty * g.th + g.th - 1, g.H - 1);
    return tile_keep(d, x0, y0, x1, y1);
}

// Position j of the emission order handles primitive i = order[j] (identity when order is NULL).
// COUNT (EMIT = false) writes the surviving count of position j into counts_or_offsets[j]; EMIT
// writes the pairs at offsets[j] in slot order r (row-major over the box).  Boxes of at most
// kSmallBox tiles are walked by their own thread; larger ones by the whole warp, 32 slots at a
// time, with ballot prefix counts keeping the pairs in r order.
//
// Thread t visits position j = (t * stride) mod n with stride coprime to n (a bijection).  Outputs are
// indexed by j, so the visiting order changes nothing but the schedule: in depth order the
// near-camera primitives with the largest boxes are neighbours, and a contiguous assignment would
// pile them onto the same few warps.
template <bool EMIT>
__global__ void __launch_bounds__(256) bin_kernel(const float *__restrict__ rec, const int4 *__restrict__ bbox,
                                                  const int *__restrict__ tcount, const int *__restrict__ order,
                                                  int64_t n, int64_t stride, Grid g,
                                                  int32_t *__restrict__ counts_or_offsets,
                                                  uint64_t *__restrict__ keys, uint32_t *__restrict__ vals) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t j = t < n ? (int64_t)(((unsigned long long)t * (unsigned long long)stride) % (unsigned long long)n)
                            : n;
    const int lane = threadIdx.x & 31;
    int i = 0, area = 0;
    int4 bb = make_int4(0, 0, 0, 0);
    if (j < n) {
        i = order ? order[j] : (int)j;
        if (tcount[i] > 0) {
            bb = bbox[i];
            bb.x = max(bb.x, 0);  // never leave the tile grid, whatever the caller's boxes say
            bb.y = max(bb.y, 0);
            bb.z = min(bb.z, g.Wt);
            bb.w = min(bb.w, g.Ht);
            const int w = bb.z - bb.x, h = bb.w - bb.y;
            area = (w > 0 && h > 0) ? w * h : 0;
        }
    }
    if (area > 0 && area <= kSmallBox) {
        const CullData d = load_cull(rec, i);
        const uint32_t depth_bits = EMIT ? __float_as_uint(rec[(size_t)i * XPR_REC_FLOATS + 9]) : 0u;
        const int64_t out = EMIT ? (int64_t)counts_or_offsets[j] : 0;
        int cnt = 0;
        for (int ty = bb.y; ty < bb.w; ++ty)
            for (int tx = bb.x; tx < bb.z; ++tx) {
                if (!keep_tile(d, g, tx, ty)) continue;
                if (EMIT) {
                    keys[out + cnt] = ((uint64_t)(uint32_t)(ty * g.Wt + tx) << 32) | depth_bits;
                    vals[out + cnt] = (uint32_t)i;
                }
                ++cnt;
            }
        if (!EMIT) counts_or_offsets[j] = cnt;
    } else if (!EMIT && j < n && area == 0) {
        counts_or_offsets[j] = 0;
    }
    unsigned big = __ballot_sync(kFullMask, area > kSmallBox);
    while (big) {
        const int src = __ffs(big) - 1;
        big &= big - 1;
        const long long jb = __shfl_sync(kFullMask, (long long)j, src);
        const int ib = __shfl_sync(kFullMask, i, src);
        const int areab = __shfl_sync(kFullMask, area, src);
        const int bx = __shfl_sync(kFullMask, bb.x, src), by = __shfl_sync(kFullMask, bb.y, src);
        const int bw = __shfl_sync(kFullMask, bb.z, src) - bx;
        const CullData d = load_cull(rec, ib);
        const uint32_t depth_bits = EMIT ? __float_as_uint(rec[(size_t)ib * XPR_REC_FLOATS + 9]) : 0u;
        const int64_t out = EMIT ? (int64_t)counts_or_offsets[jb] : 0;
        int cnt = 0;
        for (int r0 = 0; r0 < areab; r0 += 32) {
            const int r = r0 + lane;
            int tx = 0, ty = 0;
            bool keep = false;
            if (r < areab) {
                ty = by + r / bw;
                tx = bx + r % bw;
                keep = keep_tile(d, g, tx, ty);
            }
            const unsigned m = __ballot_sync(kFullMask, keep);
            if (EMIT && keep) {
                const int64_t pos = out + cnt + __popc(m & ((1u << lane) - 1u));
                keys[pos] = ((uint64_t)(uint32_t)(ty * g.Wt + tx) << 32) | depth_bits;
                vals[pos] = (uint32_t)ib;
            }
            cnt += __popc(m);
        }
        if (!EMIT && lane == 0) counts_or_offsets[jb] = cnt;
    }
}

// Sort key of the depth order: camera-z bits of primitives that have tiles, all ones otherwise
// (those go last, in index order).  Depth of a primitive with tiles is > z_near > 0, so its float
// bits order like the values.
__global__ void depth_key_kernel(const float *__restrict__ rec, const int *__restrict__ tcount, int64_t n,
                                 uint64_t *__restrict__ keys, uint32_t *__restrict__ vals) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    keys[i] = tcount[i] > 0 ? (uint64_t)__float_as_uint(rec[(size_t)i * XPR_REC_FLOATS + 9]) : 0xffffffffull;
    vals[i] = (uint32_t)i;
}

// ---- device-wide exclusive scan (three phases: block reduce, scan of block sums, block scan) ----
constexpr int kScanThreads = 512;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;

__device__ __forceinline__ int64_t block_exclusive_scan(int64_t v, int64_t *smem_warp, int64_t *total) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int64_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int64_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) smem_warp[wid] = x;
    __syncthreads();
    if (wid == 0) {
        const int nw = blockDim.x >> 5;
        int64_t w = lane < nw ? smem_warp[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int64_t y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        if (lane < nw) smem_warp[lane] = w;
    }
    __syncthreads();
    int64_t prefix = wid > 0 ? smem_warp[wid - 1] : 0;
    *total = smem_warp[(blockDim.x >> 5) - 1];
    __syncthreads();
    return prefix + x - v;
}

__global__ void __launch_bounds__(kScanThreads) scan_reduce_kernel(const int32_t *__restrict__ in, int64_t n,
                                                                   int64_t *__restrict__ partials) {
    __shared__ int64_t sw[32];
    const int64_t base = (int64_t)blockIdx.x * kScanTile;
    int64_t s = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        int64_t j = base + (int64_t)k * kScanThreads + threadIdx.x;
        if (j < n) s += in[j];
    }
    int64_t tot;
    block_exclusive_scan(s, sw, &tot);
    if (threadIdx.x == 0) partials[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(kScanThreads) scan_partials_kernel(int64_t *__restrict__ partials, int64_t nb,
                                                                     int64_t *__restrict__ total_out) {
    __shared__ int64_t sw[32];
    int64_t carry = 0;
    for (int64_t base = 0; base < nb; base += kScanThreads) {
        int64_t j = base + threadIdx.x;
        int64_t v = j < nb ? partials[j] : 0;
        int64_t tot;
        int64_t ex = block_exclusive_scan(v, sw, &tot);
        if (j < nb) partials[j] = carry + ex;
        carry += tot;
    }
    if (threadIdx.x == 0) *total_out = carry;
}

// Items are read in a blocked layout (thread t owns kScanItems consecutive items) so the
// in-place case (in == out) is safe: every item is read before it is written, by its owner.
__global__ void __launch_bounds__(kScanThreads) scan_downsweep_kernel(const int32_t *in, int32_t *out, int64_t n,
                                                                      const int64_t *__restrict__ partials,
                                                                      const int64_t *__restrict__ total) {
    __shared__ int64_t sw[32];
    const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    int32_t v[kScanItems];
    int64_t s = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        int64_t j = base + k;
        v[k] = j < n ? in[j] : 0;
        s += v[k];
    }
    int64_t tot;
    int64_t ex = block_exclusive_scan(s, sw, &tot) + partials[blockIdx.x];
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        int64_t j = base + k;
        if (j < n) out[j] = (int32_t)ex;
        ex += v[k];
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) out[n] = (int32_t)*total;
}

}  // namespace

int64_t *scan_total_ptr(void *partials, int64_t n) {
    return reinterpret_cast<int64_t *>(partials) + (n + kScanTile - 1) / kScanTile + 1;
}

size_t scan_partials_bytes(int64_t n) {
    int64_t nb = (n + kScanTile - 1) / kScanTile;
    return (size_t)((nb + 2) * sizeof(int64_t) + 255) / 256 * 256;
}

// partials layout: [nb] block sums, then the total (device int64) if total_out is NULL.
int launch_exclusive_scan(const int32_t *in, int32_t *out, int64_t n, void *partials, int64_t *total_out,
                          cudaStream_t st) {
    int64_t nb = (n + kScanTile - 1) / kScanTile;
    int64_t *part = reinterpret_cast<int64_t *>(partials);
    int64_t *tot = total_out ? total_out : scan_total_ptr(partials, n);
    if (n == 0) {
        XPR_CUDA_TRY(cudaMemsetAsync(out, 0, sizeof(int32_t), st));
        XPR_CUDA_TRY(cudaMemsetAsync(tot, 0, sizeof(int64_t), st));
        return XPR_OK;
    }
    scan_reduce_kernel<<<(unsigned)nb, kScanThreads, 0, st>>>(in, n, part);
    XPR_LAUNCH_CHECK("scan_reduce_kernel");
    scan_partials_kernel<<<1, kScanThreads, 0, st>>>(part, nb, tot);
    XPR_LAUNCH_CHECK("scan_partials_kernel");
    scan_downsweep_kernel<<<(unsigned)nb, kScanThreads, 0, st>>>(in, out, n, part, tot);
    XPR_LAUNCH_CHECK("scan_downsweep_kernel");
    return XPR_OK;
}

static Grid make_grid(const XprCamera &cam, const XprConfig &cfg) {
    Grid g;
    g.W = cam.width;
    g.H = cam.height;
    g.tw = cfg.tile_w;
    g.th = cfg.tile_h;
    g.Wt = tiles_x(cam, cfg);
    g.Ht = tiles_y(cam, cfg);
    return g;
}

// A stride coprime to n for the thread -> position bijection (a prime that does not divide n).
static int64_t visit_stride(int64_t n) {
    static const int64_t primes[] = {7919, 7927, 7933, 7937, 7949, 7951, 7963, 7993};
    for (int64_t p : primes)
        if (n % p != 0) return p % n == 0 ? 1 : p;
    return 1;  // n is a multiple of every listed prime (impossible for n < 2^31): contiguous visiting
}

int launch_bin_count(const float *rec, const int32_t *bbox, const int32_t *tc, const int32_t *order, int64_t n,
                     const XprCamera &cam, const XprConfig &cfg, int32_t *counts, cudaStream_t st) {
    if (n == 0) return XPR_OK;
    const int tpb = 256;
    bin_kernel<false><<<(unsigned)((n + tpb - 1) / tpb), tpb, 0, st>>>(
        rec, reinterpret_cast<const int4 *>(bbox), tc, order, n, visit_stride(n), make_grid(cam, cfg), counts,
        nullptr, nullptr);
    XPR_LAUNCH_CHECK("bin_count_kernel");
    return XPR_OK;
}

int launch_bin_emit(const float *rec, const int32_t *bbox, const int32_t *tc, const int32_t *order, int64_t n,
                    const XprCamera &cam, const XprConfig &cfg, const int32_t *offsets, uint64_t *keys,
                    uint32_t *vals, cudaStream_t st) {
    if (n == 0) return XPR_OK;
    const int tpb = 256;
    bin_kernel<true><<<(unsigned)((n + tpb - 1) / tpb), tpb, 0, st>>>(
        rec, reinterpret_cast<const int4 *>(bbox), tc, order, n, visit_stride(n), make_grid(cam, cfg),
        const_cast<int32_t *>(offsets), keys, vals);
    XPR_LAUNCH_CHECK("bin_emit_kernel");
    return XPR_OK;
}

size_t depth_order_workspace_bytes(int64_t n) {
    const size_t a = ((size_t)n * 8 + 255) / 256 * 256, b = ((size_t)n * 4 + 255) / 256 * 256;
    return 2 * a + b + 256 + sort_workspace_bytes(n, 1);
}

int launch_depth_order(const float *rec, const int32_t *tc, int64_t n, int32_t *order, void *ws, size_t ws_bytes,
                       cudaStream_t st) {
    if (n == 0) return XPR_OK;
    if (ws_bytes < depth_order_workspace_bytes(n))
        return fail(XPR_ERR_INVALID, "xpr_depth_order: workspace %zu < %zu bytes", ws_bytes,
                    depth_order_workspace_bytes(n));
    const size_t a = ((size_t)n * 8 + 255) / 256 * 256, b = ((size_t)n * 4 + 255) / 256 * 256;
    char *p = reinterpret_cast<char *>(ws);
    uint64_t *keys = reinterpret_cast<uint64_t *>(p);
    uint64_t *keys_sorted = reinterpret_cast<uint64_t *>(p + a);
    uint32_t *vals = reinterpret_cast<uint32_t *>(p + 2 * a);
    int32_t *ranges = reinterpret_cast<int32_t *>(p + 2 * a + b);
    void *sort_ws = p + 2 * a + b + 256;
    depth_key_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(rec, tc, n, keys, vals);
    XPR_LAUNCH_CHECK("depth_key_kernel");
    return launch_sort(keys, vals, n, 1, 0, keys_sorted, reinterpret_cast<uint32_t *>(order), ranges, sort_ws,
                       sort_workspace_bytes(n, 1), st);
}

}  // namespace xpr
