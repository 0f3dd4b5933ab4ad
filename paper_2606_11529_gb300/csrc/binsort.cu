// Rasterizer, both halves fused (Sec. 4.2 "Replicate, Assign tile ID, Cull" + "Sort and identify
// bounds"): the per-tile lists are built directly in their sorted order, with no key array and no
// radix passes.
//
// Input: the records in emission (depth) order, order[] from xpr_depth_order.  Wanted: for every
// tile, the kept records in that order, i.e. a stable counting sort of the (record, tile) pairs by
// tile.  The pairs of one record fall on distinct tiles, so a warp that walks records one after
// another can rank pairs with private per-tile counters and no conflict resolution:
//
//   * tile rows are grouped into bands of BR rows; a work unit is (band, range of consecutive
//     emission positions) and owns one counter per tile of its band in shared memory;
//   * the unit's warp walks its positions in order; for each record whose box meets the band, the
//     lanes take the box's band slots 32 at a time (all on different tiles), apply the exact FP32
//     cull of cull.cuh and bump the counter of each kept tile;
//   * count pass: the counters are stored as the unit's row of a (unit x band tile) matrix; then
//     for each tile, an exclusive prefix over the tiles before it and over the band's units before
//     this one turns each entry into the output position of the unit's first pair on that tile,
//     and gives the tile ranges [start, end) directly;
//   * emit pass: the same walk with the counters started at those positions writes
//     vals[counter++] = record index.
// Within a tile, units come in position order and a unit's pairs in walk order, so the result is
// the (tile, depth, index) order of the key sort, bit for bit, with the same kept set.
//
// Work balance.  The cost of a walk is about (band slots + a per-record overhead) summed over the
// records met, and it is very uneven: near the camera one record covers hundreds of tiles.  So the
// positions are first cut into chunks of Q positions; for every (band, chunk) the cost is summed;
// a work quantum E is chosen on the device from the total so that the units fit a fixed budget;
// and each (band, chunk) becomes floor(cost / E) + 1 units, cut where its running cost crosses a
// multiple of E.  A unit therefore walks at most Q positions and about E slots.  Each band's
// units are padded to a multiple of 32 (empty units) so the column prefix works on 32-row
// segments that never straddle two bands.
#include "cull.cuh"

namespace xpr {
namespace {

constexpr int kUnitWarps = 8;     // warps (units) per walk block
constexpr int kColThreads = 256;
constexpr int kSeg = 32;          // units per column-scan segment (and band padding granule)
constexpr int kKappa = 32;        // per-record cost of a walk, in slot units
constexpr int kMinQuantum = 2048; // smallest work quantum E, in slot units
constexpr int kMaxBandCols = 6400;
constexpr int kWalkSmemMax = kUnitWarps * kMaxBandCols * 4;  // 204800 B: one band row per warp
constexpr int kPlanThreads = 1024;
constexpr int kMaxBands = 2048;   // views x bands taken (the unit budget is sized for it)

struct Shape {
    int64_t n;       // records per view
    int V;           // views
    Grid g;
    int BR;          // tile rows per band
    int nb;          // bands per view
    int bt;          // band row stride of the matrix: BR * Wt
    int T1;          // tiles per view
    int64_t Q;       // positions per chunk
    int npc;         // chunks per view
    int max_units;   // unit budget (matrix rows)
};

Shape make_shape(int64_t n, int V, const XprCamera &cam, const XprConfig &cfg) {
    Shape s;
    s.n = n;
    s.V = V;
    s.g = make_grid(cam, cfg);
    s.BR = max(1, min(8, 2048 / s.g.Wt));
    s.nb = (s.g.Ht + s.BR - 1) / s.BR;
    s.bt = s.BR * s.g.Wt;
    s.T1 = s.g.Wt * s.g.Ht;
    s.max_units = 12288 * min(V, 4);
    // at most half the budget goes to the one-unit-per-(band, chunk) minimum
    const int64_t vb = (int64_t)V * s.nb;
    int64_t npc_cap = max((int64_t)1, (int64_t)(s.max_units / 2) / vb);
    int64_t Q = max((int64_t)4096, (n + npc_cap - 1) / npc_cap);
    Q = (Q + 31) / 32 * 32;
    s.Q = Q;
    s.npc = (int)((n + Q - 1) / Q);
    // the band padding can add up to kSeg - 1 units per band
    s.max_units += (int)(vb * kSeg);
    return s;
}

inline size_t al256(size_t b) { return (b + 255) / 256 * 256; }

struct Plan {
    unsigned long long h_total;  // sum of all (band, chunk) costs
    long long quantum;           // work quantum E
    long long units;             // units in use (a multiple of kSeg)
    long long pad;
};

struct Ws {
    int2 *box;        // [V n] packed boxes in emission order
    int32_t *cost;    // [V nb npc] (band, chunk) cost sums, band-major
    int32_t *lofs;    // [V nb npc] first unit of a (band, chunk) within its band
    int32_t *bandu;   // [V nb] units per band (padded), then the first unit of each band
    int4 *desc;       // [max_units] (band, chunk, sub-unit, sub-units); chunk -1: padding
    int32_t *ustart;  // [max_units] first position of sub-unit s >= 1
    Plan *plan;
    int32_t *mat;     // [max_units][bt] counts, then first output positions
    int32_t *part;    // [max_units / kSeg][bt] segment sums, then segment prefixes
    int32_t *tot;     // [V T1] tile totals
    int32_t *start;   // [V T1 + 1] tile starts
    void *scan_tiles; // scan partials over V T1 entries
    void *scan_bands; // scan partials over V nb entries
};

size_t carve(const Shape &s, void *base, Ws *w) {
    const int64_t nr = s.n * s.V, nt = (int64_t)s.T1 * s.V, vb = (int64_t)s.V * s.nb;
    const int64_t ncost = vb * s.npc;
    size_t off = 0;
    char *p = reinterpret_cast<char *>(base);
    auto take = [&](size_t bytes) {
        char *q = p ? p + off : nullptr;
        off += al256(bytes);
        return q;
    };
    char *a = take((size_t)nr * sizeof(int2));
    char *b = take((size_t)ncost * 4);
    char *c = take((size_t)ncost * 4);
    char *d = take((size_t)(vb + 1) * 4);
    char *e = take((size_t)s.max_units * sizeof(int4));
    char *f = take((size_t)s.max_units * 4);
    char *g = take(sizeof(Plan));
    char *h = take((size_t)s.max_units * s.bt * 4);
    char *i = take((size_t)(s.max_units / kSeg) * s.bt * 4);
    char *j = take((size_t)nt * 4);
    char *k = take((size_t)(nt + 1) * 4);
    char *l = take(scan_partials_bytes(nt));
    char *m = take(scan_partials_bytes(vb));
    if (w) {
        w->box = reinterpret_cast<int2 *>(a);
        w->cost = reinterpret_cast<int32_t *>(b);
        w->lofs = reinterpret_cast<int32_t *>(c);
        w->bandu = reinterpret_cast<int32_t *>(d);
        w->desc = reinterpret_cast<int4 *>(e);
        w->ustart = reinterpret_cast<int32_t *>(f);
        w->plan = reinterpret_cast<Plan *>(g);
        w->mat = reinterpret_cast<int32_t *>(h);
        w->part = reinterpret_cast<int32_t *>(i);
        w->tot = reinterpret_cast<int32_t *>(j);
        w->start = reinterpret_cast<int32_t *>(k);
        w->scan_tiles = l;
        w->scan_bands = m;
    }
    return off;
}

// ---------------------------------------------------------------------------------------------
// box[j] = the tile box of record order[j], clamped to the grid, packed x0 | x1 << 16, y0 | y1 << 16
// (empty when the record has no tiles).
__global__ void gather_box_kernel(const int4 *__restrict__ bbox, const int32_t *__restrict__ tcount,
                                  const int32_t *__restrict__ order, int64_t nr, Grid g, int2 *__restrict__ box) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= nr) return;
    const int i = order[j];
    int2 out = make_int2(0, 0);
    if (tcount[i] > 0) {
        int4 bb = bbox[i];
        bb.x = max(bb.x, 0);
        bb.y = max(bb.y, 0);
        bb.z = min(bb.z, g.Wt);
        bb.w = min(bb.w, g.Ht);
        if (bb.z > bb.x && bb.w > bb.y) out = make_int2(bb.x | (bb.z << 16), bb.y | (bb.w << 16));
    }
    box[j] = out;
}

struct Box {
    int x0, x1, y0, y1;
};

__device__ __forceinline__ Box unpack(int2 b) {
    return Box{b.x & 0xffff, b.x >> 16, b.y & 0xffff, b.y >> 16};
}

// Walk cost of a box on band rows [r0, r1): its slots there plus the per-record overhead (0 if
// the box misses the band or is empty).
__device__ __forceinline__ int band_cost(const Box &b, int r0, int r1) {
    const int y0 = max(b.y0, r0), y1 = min(b.y1, r1);
    return (b.x1 > b.x0 && y1 > y0) ? (y1 - y0) * (b.x1 - b.x0) + kKappa : 0;
}

// One warp per (view, chunk): the walk cost of each band over the chunk's positions.
__global__ void __launch_bounds__(256) chunk_cost_kernel(const int2 *__restrict__ box, Shape s,
                                                         int32_t *__restrict__ cost, Plan *__restrict__ plan) {
    extern __shared__ int32_t s_acc[];  // [8 warps][nb]
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t wid = (int64_t)blockIdx.x * 8 + warp;
    if (wid >= (int64_t)s.V * s.npc) return;
    const int64_t v = wid / s.npc, pc = wid - v * s.npc;
    int32_t *acc = s_acc + warp * s.nb;
    for (int b = lane; b < s.nb; b += 32) acc[b] = 0;
    __syncwarp();
    const int64_t jb = v * s.n + pc * s.Q, je = v * s.n + min((pc + 1) * s.Q, s.n);
    for (int64_t j0 = jb; j0 < je; j0 += 32) {
        const int64_t j = j0 + lane;
        const Box b = j < je ? unpack(box[j]) : Box{0, 0, 0, 0};
        const bool has = b.x1 > b.x0;
        const int blo = __reduce_min_sync(kFullMask, has ? (unsigned)(b.y0 / s.BR) : 0x7fffffffu);
        const int bhi = (int)__reduce_max_sync(kFullMask, has ? (unsigned)((b.y1 - 1) / s.BR) : 0u);
        for (int band = blo; band <= bhi; ++band) {
            const int c = band_cost(b, band * s.BR, min(band * s.BR + s.BR, s.g.Ht));
            const int sum = (int)__reduce_add_sync(kFullMask, (unsigned)c);
            if (lane == 0) acc[band] += sum;
        }
    }
    __syncwarp();
    unsigned long long mine = 0;
    for (int b = lane; b < s.nb; b += 32) {
        cost[((int64_t)v * s.nb + b) * s.npc + pc] = acc[b];
        mine += (unsigned long long)acc[b];
    }
    for (int o = 16; o > 0; o >>= 1) mine += __shfl_xor_sync(kFullMask, mine, o);
    if (lane == 0) atomicAdd(&plan->h_total, mine);
}

__device__ __forceinline__ long long plan_quantum(const Plan *plan, const Shape &s) {
    const long long vb = (long long)s.V * s.nb;
    const long long avail = (long long)s.max_units - vb * kSeg - vb * s.npc;  // > 0 by the shape
    const long long q = ((long long)plan->h_total + avail - 1) / (avail > 0 ? avail : 1);
    return q > kMinQuantum ? q : kMinQuantum;
}

// One block per band: units of each (band, chunk) = floor(cost / E) + 1, their first unit within
// the band (block-wide exclusive scan), and the band's unit count padded to a multiple of kSeg.
__global__ void __launch_bounds__(kPlanThreads) plan_band_kernel(const int32_t *__restrict__ cost, Shape s,
                                                                 const Plan *__restrict__ plan,
                                                                 int32_t *__restrict__ lofs,
                                                                 int32_t *__restrict__ bandu) {
    __shared__ int s_warp[kPlanThreads / 32];
    __shared__ int s_carry;
    const int64_t vb = blockIdx.x;
    const long long E = plan_quantum(plan, s);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (threadIdx.x == 0) s_carry = 0;
    __syncthreads();
    for (int base = 0; base < s.npc; base += kPlanThreads) {
        const int pc = base + threadIdx.x;
        const int u = pc < s.npc ? (int)(cost[vb * s.npc + pc] / E) + 1 : 0;
        int x = u;
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(kFullMask, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) s_warp[wid] = x;
        __syncthreads();
        if (wid == 0) {
            int w = s_warp[lane];
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(kFullMask, w, o);
                if (lane >= o) w += y;
            }
            s_warp[lane] = w;
        }
        __syncthreads();
        const int excl = s_carry + (wid > 0 ? s_warp[wid - 1] : 0) + x - u;
        if (pc < s.npc) lofs[vb * s.npc + pc] = excl;
        __syncthreads();
        if (threadIdx.x == 0) s_carry += s_warp[kPlanThreads / 32 - 1];
        __syncthreads();
    }
    if (threadIdx.x == 0) bandu[vb] = (s_carry + kSeg - 1) / kSeg * kSeg;
}

// One block per band (after the band scan turned bandu into first units): unit descriptors.
__global__ void __launch_bounds__(256) describe_units_kernel(const int32_t *__restrict__ cost,
                                                             const int32_t *__restrict__ lofs,
                                                             const int32_t *__restrict__ bandfirst, Shape s,
                                                             Plan *__restrict__ plan, int4 *__restrict__ desc) {
    const int vb = blockIdx.x;
    const long long E = plan_quantum(plan, s);
    const int first = bandfirst[vb], last = bandfirst[vb + 1];
    const int used = s.npc > 0 ? lofs[(int64_t)vb * s.npc + s.npc - 1] +
                                     (int)(cost[(int64_t)vb * s.npc + s.npc - 1] / E) + 1
                               : 0;
    for (int pc = threadIdx.x; pc < s.npc; pc += blockDim.x) {
        const int nsub = (int)(cost[(int64_t)vb * s.npc + pc] / E) + 1;
        const int u0 = first + lofs[(int64_t)vb * s.npc + pc];
        for (int k = 0; k < nsub; ++k) desc[u0 + k] = make_int4(vb, pc, k, nsub);
    }
    for (int u = first + used + threadIdx.x; u < last; u += blockDim.x) desc[u] = make_int4(vb, -1, 0, 0);
    if (vb == (int)gridDim.x - 1 && threadIdx.x == 0) {
        plan->quantum = E;
        plan->units = last;
    }
}

// One warp per (view, chunk): where each (band, chunk)'s sub-units s >= 1 begin, i.e. the first
// position after the running cost crosses s * E.
__global__ void __launch_bounds__(256) cut_units_kernel(const int2 *__restrict__ box, Shape s,
                                                        const int32_t *__restrict__ lofs,
                                                        const int32_t *__restrict__ bandfirst,
                                                        const int32_t *__restrict__ cost,
                                                        const Plan *__restrict__ plan,
                                                        int32_t *__restrict__ ustart) {
    extern __shared__ int32_t s_run[];  // [8 warps][nb] running cost
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t wid = (int64_t)blockIdx.x * 8 + warp;
    if (wid >= (int64_t)s.V * s.npc) return;
    const int64_t v = wid / s.npc, pc = wid - v * s.npc;
    const long long E = plan->quantum;
    int32_t *run = s_run + warp * s.nb;
    for (int b = lane; b < s.nb; b += 32) run[b] = 0;
    __syncwarp();
    const int64_t jv = v * s.n;
    const int64_t jb = jv + pc * s.Q, je = jv + min((pc + 1) * s.Q, s.n);
    for (int64_t j0 = jb; j0 < je; j0 += 32) {
        const int64_t j = j0 + lane;
        const Box b = j < je ? unpack(box[j]) : Box{0, 0, 0, 0};
        const bool has = b.x1 > b.x0;
        const int blo = __reduce_min_sync(kFullMask, has ? (unsigned)(b.y0 / s.BR) : 0x7fffffffu);
        const int bhi = (int)__reduce_max_sync(kFullMask, has ? (unsigned)((b.y1 - 1) / s.BR) : 0u);
        for (int band = blo; band <= bhi; ++band) {
            const int c = band_cost(b, band * s.BR, min(band * s.BR + s.BR, s.g.Ht));
            int incl = c;
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(kFullMask, incl, o);
                if (lane >= o) incl += y;
            }
            const int r = run[band];
            __syncwarp();
            if (c > 0) {
                const long long lo = (long long)(r + incl - c) / E, hi = (long long)(r + incl) / E;
                if (hi > lo) {
                    const int64_t vbi = v * s.nb + band;
                    const int u0 = bandfirst[vbi] + lofs[vbi * s.npc + pc];
                    const int nsub = (int)(cost[vbi * s.npc + pc] / E) + 1;
                    for (long long k = lo + 1; k <= hi && k < nsub; ++k) ustart[u0 + k] = (int32_t)(j + 1 - jv);
                }
            }
            if (lane == 31) run[band] = r + incl;
            __syncwarp();
        }
    }
}

// One warp per unit; EMIT = false counts, EMIT = true writes.
template <bool EMIT>
__global__ void __launch_bounds__(kUnitWarps * 32) walk_kernel(const float *__restrict__ rec,
                                                               const int32_t *__restrict__ order,
                                                               const int2 *__restrict__ box, Shape s,
                                                               const int4 *__restrict__ desc,
                                                               const int32_t *__restrict__ ustart,
                                                               const Plan *__restrict__ plan,
                                                               int32_t *__restrict__ mat,
                                                               uint32_t *__restrict__ vals) {
    extern __shared__ int32_t s_ctr[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t u = (int64_t)blockIdx.x * kUnitWarps + warp;
    if (u >= plan->units) return;
    const int4 d = desc[u];  // (view * nb + band, chunk or -1, sub-unit, sub-units)
    const int v = d.x / s.nb, band = d.x - v * s.nb;
    const int Wt = s.g.Wt;
    const int r0 = band * s.BR, r1 = min(r0 + s.BR, s.g.Ht);
    const int band_tiles = (r1 - r0) * Wt;
    int32_t *ctr = s_ctr + warp * s.bt;
    int32_t *mrow = mat + u * s.bt;
    for (int k = lane; k < band_tiles; k += 32) ctr[k] = EMIT ? mrow[k] : 0;
    __syncwarp();
    if (d.y >= 0) {
        const int64_t jv = (int64_t)v * s.n;
        const int64_t cs = (int64_t)d.y * s.Q, ce = min(cs + s.Q, s.n);
        // sub-unit bounds lie in [cs, ce] by construction; the clamps keep every read in the chunk
        const int64_t ub = d.z == 0 ? cs : min(max((int64_t)ustart[u], cs), ce);
        const int64_t ue = d.z == d.w - 1 ? ce : min(max((int64_t)ustart[u + 1], ub), ce);
        const int64_t jb = jv + ub, je = jv + ue;
        for (int64_t j0 = jb; j0 < je; j0 += 32) {
            const int64_t j = j0 + lane;
            Box b = Box{0, 0, 0, 0};
            int i = 0;
            if (j < je) {
                b = unpack(box[j]);
                i = order[j];
            }
            const bool hit = b.x1 > b.x0 && b.y0 < r1 && b.y1 > r0;
            unsigned m = __ballot_sync(kFullMask, hit);
            if (!m) continue;
            CullData cd = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, -1.f};
            if (hit) cd = load_cull(rec, i);
            while (m) {
                const int src = __ffs(m) - 1;
                m &= m - 1;
                const CullData e = shfl_cull(cd, src);
                const int is = __shfl_sync(kFullMask, i, src);
                const int x0 = __shfl_sync(kFullMask, b.x0, src), x1 = __shfl_sync(kFullMask, b.x1, src);
                const int y0 = max(__shfl_sync(kFullMask, b.y0, src), r0);
                const int y1 = min(__shfl_sync(kFullMask, b.y1, src), r1);
                const int bw = x1 - x0, area = (y1 - y0) * bw;
                SlotWalk sw(x0, y0, bw, lane);
                for (int r = 0; r < area; r += 32) {
                    if (r + lane < area && keep_tile(e, s.g, sw.tx, sw.ty)) {
                        const int k = (sw.ty - r0) * Wt + sw.tx;  // distinct across the lanes of one step
                        const int c = ctr[k];
                        ctr[k] = c + 1;
                        if (EMIT) vals[c] = (uint32_t)is;
                    }
                    sw.step();
                }
                __syncwarp();  // the next record's lanes read what this one's lanes wrote
            }
        }
    }
    if (!EMIT) {
        __syncwarp();
        for (int k = lane; k < band_tiles; k += 32) mrow[k] = ctr[k];
    }
}

__device__ __forceinline__ int band_tiles_of(const Shape &s, int vb) {
    const int band = vb % s.nb;
    const int r0 = band * s.BR, r1 = min(r0 + s.BR, s.g.Ht);
    return (r1 - r0) * s.g.Wt;
}

// part[seg][k] = sum of column k over the kSeg units of segment seg (a segment lies in one band).
__global__ void __launch_bounds__(kColThreads) colsum_kernel(const int32_t *__restrict__ mat, Shape s,
                                                             const int4 *__restrict__ desc,
                                                             const Plan *__restrict__ plan,
                                                             int32_t *__restrict__ part) {
    const int64_t seg = blockIdx.y;
    if (seg * kSeg >= plan->units) return;
    const int k = blockIdx.x * kColThreads + threadIdx.x;
    if (k >= band_tiles_of(s, desc[seg * kSeg].x)) return;
    const int32_t *m = mat + seg * kSeg * (int64_t)s.bt + k;
    int sum = 0;
#pragma unroll 8
    for (int r = 0; r < kSeg; ++r) sum += m[(int64_t)r * s.bt];
    part[seg * (int64_t)s.bt + k] = sum;
}

// Per band and column: exclusive prefix over the band's segments (in place) and the tile total.
__global__ void __launch_bounds__(kColThreads) segscan_kernel(int32_t *__restrict__ part, Shape s,
                                                              const int32_t *__restrict__ bandfirst,
                                                              int32_t *__restrict__ tot) {
    const int vb = blockIdx.y;
    const int k = blockIdx.x * kColThreads + threadIdx.x;
    if (k >= band_tiles_of(s, vb)) return;
    const int64_t g0 = bandfirst[vb] / kSeg, g1 = bandfirst[vb + 1] / kSeg;
    int run = 0;
    for (int64_t g = g0; g < g1; ++g) {
        int32_t *p = part + g * (int64_t)s.bt + k;
        const int x = *p;
        *p = run;
        run += x;
    }
    const int v = vb / s.nb, band = vb - v * s.nb;
    tot[(int64_t)v * s.T1 + (int64_t)band * s.BR * s.g.Wt + k] = run;
}

// Matrix entries -> first output position of the (unit, tile); a band's first segment also
// writes the tile ranges (an empty tile gets [0, 0), as from the key sort's segment search).
__global__ void __launch_bounds__(kColThreads) apply_kernel(int32_t *__restrict__ mat, const int32_t *__restrict__ part,
                                                            const int32_t *__restrict__ start, Shape s,
                                                            const int4 *__restrict__ desc,
                                                            const int32_t *__restrict__ bandfirst,
                                                            const Plan *__restrict__ plan, int2 *__restrict__ ranges) {
    const int64_t seg = blockIdx.y;
    if (seg * kSeg >= plan->units) return;
    const int vb = desc[seg * kSeg].x;
    const int k = blockIdx.x * kColThreads + threadIdx.x;
    if (k >= band_tiles_of(s, vb)) return;
    const int v = vb / s.nb, band = vb - v * s.nb;
    const int64_t gt = (int64_t)v * s.T1 + (int64_t)band * s.BR * s.g.Wt + k;
    if (seg * kSeg == bandfirst[vb]) {
        const int a = start[gt], b = start[gt + 1];
        ranges[gt] = b > a ? make_int2(a, b) : make_int2(0, 0);
    }
    int run = start[gt] + part[seg * (int64_t)s.bt + k];
    int32_t *m = mat + seg * kSeg * (int64_t)s.bt + k;
    for (int r = 0; r < kSeg; ++r) {
        const int x = m[(int64_t)r * s.bt];
        m[(int64_t)r * s.bt] = run;
        run += x;
    }
}

}  // namespace

size_t binsort_workspace_bytes(int64_t n, int n_views, const XprCamera &cam, const XprConfig &cfg) {
    return carve(make_shape(n, n_views, cam, cfg), nullptr, nullptr);
}

bool binsort_supported(const XprCamera &cam, const XprConfig &cfg, int n_views) {
    const Grid g = make_grid(cam, cfg);
    // packed 16-bit box coordinates; one band row of counters per warp fits (<= 200 KB per block);
    // the unit budget holds at least two units per (band, chunk) for every band of every view
    if (g.Wt > kMaxBandCols || g.Ht >= 32768) return false;
    const int BR = max(1, min(8, 2048 / g.Wt));
    return (int64_t)n_views * ((g.Ht + BR - 1) / BR) <= kMaxBands;
}

int launch_binsort(const float *rec, const int32_t *bbox, const int32_t *tc, const int32_t *order, int64_t n,
                   int n_views, const XprCamera &cam, const XprConfig &cfg, int32_t *ranges, uint32_t *vals,
                   int64_t capacity, int64_t *n_isect, void *ws, size_t ws_bytes, cudaStream_t st) {
    const Shape s = make_shape(n, n_views, cam, cfg);
    Ws w;
    const size_t need = carve(s, ws, &w);
    if (ws_bytes < need) return fail(XPR_ERR_INVALID, "xpr_bin_sorted: workspace %zu < %zu bytes", ws_bytes, need);
    const int64_t nr = n * n_views, nt = (int64_t)s.T1 * n_views, vb = (int64_t)n_views * s.nb;
    if ((int64_t)s.Q * (s.bt + kKappa) > 0x7fffffffLL)
        return fail(XPR_ERR_INVALID, "xpr_bin_sorted: %lld records per view are too many", (long long)n);
    *n_isect = 0;
    if (nr == 0) {
        XPR_CUDA_TRY(cudaMemsetAsync(ranges, 0, (size_t)nt * 2 * sizeof(int32_t), st));
        return XPR_OK;
    }
    const size_t smem = (size_t)kUnitWarps * s.bt * sizeof(int32_t);
    if (smem > (size_t)kWalkSmemMax) return fail(XPR_ERR_INVALID, "xpr_bin_sorted: %zu bytes of counters", smem);
    // One fixed limit for every call: concurrent callers (other host threads, other grid sizes) must
    // never lower it below what a launch in flight on another stream was checked against.
    XPR_CUDA_TRY(cudaFuncSetAttribute(walk_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, kWalkSmemMax));
    XPR_CUDA_TRY(cudaFuncSetAttribute(walk_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, kWalkSmemMax));
    XPR_CUDA_TRY(cudaMemsetAsync(w.plan, 0, sizeof(Plan), st));

    gather_box_kernel<<<(unsigned)((nr + 255) / 256), 256, 0, st>>>(reinterpret_cast<const int4 *>(bbox), tc, order,
                                                                     nr, s.g, w.box);
    XPR_LAUNCH_CHECK("gather_box_kernel");
    const unsigned chunk_blocks = (unsigned)(((int64_t)n_views * s.npc + 7) / 8);
    const size_t band_smem = (size_t)8 * s.nb * sizeof(int32_t);
    chunk_cost_kernel<<<chunk_blocks, 256, band_smem, st>>>(w.box, s, w.cost, w.plan);
    XPR_LAUNCH_CHECK("chunk_cost_kernel");
    plan_band_kernel<<<(unsigned)vb, kPlanThreads, 0, st>>>(w.cost, s, w.plan, w.lofs, w.bandu);
    XPR_LAUNCH_CHECK("plan_band_kernel");
    int r = launch_exclusive_scan(w.bandu, w.bandu, vb, w.scan_bands, nullptr, st);
    if (r) return r;
    describe_units_kernel<<<(unsigned)vb, 256, 0, st>>>(w.cost, w.lofs, w.bandu, s, w.plan, w.desc);
    XPR_LAUNCH_CHECK("describe_units_kernel");
    cut_units_kernel<<<chunk_blocks, 256, band_smem, st>>>(w.box, s, w.lofs, w.bandu, w.cost, w.plan, w.ustart);
    XPR_LAUNCH_CHECK("cut_units_kernel");

    const unsigned walk_blocks = (unsigned)(s.max_units / kUnitWarps);
    walk_kernel<false><<<walk_blocks, kUnitWarps * 32, smem, st>>>(rec, order, w.box, s, w.desc, w.ustart, w.plan,
                                                                   w.mat, nullptr);
    XPR_LAUNCH_CHECK("walk_kernel<count>");
    const dim3 cgrid((unsigned)((s.bt + kColThreads - 1) / kColThreads), (unsigned)(s.max_units / kSeg));
    colsum_kernel<<<cgrid, kColThreads, 0, st>>>(w.mat, s, w.desc, w.plan, w.part);
    XPR_LAUNCH_CHECK("colsum_kernel");
    segscan_kernel<<<dim3(cgrid.x, (unsigned)vb), kColThreads, 0, st>>>(w.part, s, w.bandu, w.tot);
    XPR_LAUNCH_CHECK("segscan_kernel");
    if ((r = launch_exclusive_scan(w.tot, w.start, nt, w.scan_tiles, nullptr, st))) return r;
    apply_kernel<<<cgrid, kColThreads, 0, st>>>(w.mat, w.part, w.start, s, w.desc, w.bandu, w.plan,
                                                reinterpret_cast<int2 *>(ranges));
    XPR_LAUNCH_CHECK("apply_kernel");
    int64_t total = 0;
    XPR_CUDA_TRY(cudaMemcpyAsync(&total, scan_total_ptr(w.scan_tiles, nt), sizeof(int64_t), cudaMemcpyDeviceToHost,
                                 st));
    XPR_CUDA_TRY(cudaStreamSynchronize(st));
    *n_isect = total;
    if (total > 0x7fffffffLL)
        return fail(XPR_ERR_CAPACITY, "xpr_bin_sorted: %lld intersections exceed 2^31-1", (long long)total);
    if (total > capacity)
        return fail(XPR_ERR_CAPACITY, "xpr_bin_sorted: %lld intersections > capacity %lld", (long long)total,
                    (long long)capacity);
    if (total == 0) return XPR_OK;
    if (!vals) return fail(XPR_ERR_INVALID, "xpr_bin_sorted: NULL vals");
    walk_kernel<true><<<walk_blocks, kUnitWarps * 32, smem, st>>>(rec, order, w.box, s, w.desc, w.ustart, w.plan,
                                                                  w.mat, vals);
    XPR_LAUNCH_CHECK("walk_kernel<emit>");
    return XPR_OK;
}

}  // namespace xpr
