// StopThePop tile cull of Listing 1 tile_cull in row form, shared by the projection kernel (which
// counts the kept tiles of each primitive), the emit kernel (which writes them) and the fused
// bin + sort walk.  All of them must take identical decisions, so the decision is made in FP32
// with one correctly rounded IEEE operation per step (explicit __f*_rn intrinsics, no
// contraction) on the stored float32 record values.
//
// A tile is kept iff the largest response o exp(-q/2), q = d^T conic d, d = p - mu_2D, over its
// pixels reaches alpha_t, i.e. min over the tile of q <= T = 2 ln(o / alpha_t).  Inside one tile
// row (pixel rows [y0, y1]) that holds exactly for the tiles whose pixel columns meet the
// x-extent [xa, xb] of E ∩ strip, E = {q <= T}: E ∩ strip is convex, so its x-extent is one
// interval, bounded by the leftmost / rightmost point of E when that point's y lies in the strip
// and otherwise by where the boundary of E crosses y = y0 or y = y1.  With conic [[a, b], [b, c]]
// and det = ac - b^2:
//   leftmost / rightmost points:  (mx -/+ ex, my +/- sb),  ex = sqrt(T c / det),
//                                 sb = b sqrt(T / (c det));
//   crossings with y = Y:          x = mx + (-b dY -/+ sqrt(a T - det dY^2)) / a,  dY = Y - my.
// One evaluation per tile row instead of one per tile.  Tile k spans pixel columns
// [k w, k w + w - 1] (the last one clamped to W - 1), so it is kept iff
// ceil((xa + 1) / w) - 1 <= k <= floor(xb / w), and a span starting right of the image or
// ending left of it keeps nothing.
// 3DGUT evaluates pixel (x, y) at its centre (x + 0.5, y + 0.5), and its tile_cull extends the
// tile's max bounds by one pixel (ray offset): with ext = 1 the tile rows are [y0, y1 + 1], the
// columns [k w, k w + w - 1 + 1], so k >= ceil(xa / w) - 1, and the image ends at W - 1 + 1.
#pragma once

#include "xpr_internal.cuh"

namespace xpr {

struct CullData {
    float mx, my, b, det, aT, ia, ex, yl, yr, T;
};

struct Grid {
    int W, H, tw, th, Wt, Ht;
    int ext;  // ray offset of the tile's max bounds: 0 (3DGS) or 1 (3DGUT)
};

constexpr unsigned kFullMask = 0xffffffffu;
constexpr int kSmallBox = 16;  // boxes with more tiles than this are walked by a whole warp

// Per-primitive quantities of the row form, from the record's mu_2D, conic and ln_thr.
__device__ __forceinline__ CullData make_cull(float mx, float my, float a, float b, float c, float lt) {
    CullData d;
    d.mx = mx;
    d.my = my;
    d.b = b;
    d.T = __fadd_rn(lt, lt);
    d.det = __fsub_rn(__fmul_rn(a, c), __fmul_rn(b, b));
    d.aT = __fmul_rn(a, d.T);
    d.ia = __frcp_rn(a);
    d.ex = __fsqrt_rn(__fdiv_rn(__fmul_rn(d.T, c), d.det));
    const float sb = __fmul_rn(b, __fsqrt_rn(__fdiv_rn(d.T, __fmul_rn(c, d.det))));
    d.yl = __fadd_rn(my, sb);
    d.yr = __fsub_rn(my, sb);
    return d;
}

__device__ __forceinline__ CullData load_cull(const float *__restrict__ rec, int64_t i) {
    const float4 *p = reinterpret_cast<const float4 *>(rec + (size_t)i * XPR_REC_FLOATS);
    const float4 a = __ldg(p), b = __ldg(p + 1), c = __ldg(p + 2);
    return make_cull(a.x, a.y, a.z, a.w, b.x, c.z);
}

__device__ __forceinline__ CullData shfl_cull(const CullData &d, int src) {
    CullData e;
    e.mx = __shfl_sync(kFullMask, d.mx, src);
    e.my = __shfl_sync(kFullMask, d.my, src);
    e.b = __shfl_sync(kFullMask, d.b, src);
    e.det = __shfl_sync(kFullMask, d.det, src);
    e.aT = __shfl_sync(kFullMask, d.aT, src);
    e.ia = __shfl_sync(kFullMask, d.ia, src);
    e.ex = __shfl_sync(kFullMask, d.ex, src);
    e.yl = __shfl_sync(kFullMask, d.yl, src);
    e.yr = __shfl_sync(kFullMask, d.yr, src);
    e.T = __shfl_sync(kFullMask, d.T, src);
    return e;
}

// Kept tile columns [ka, kb] of tile row ty (unclamped to any box); false if none.
__device__ __forceinline__ bool row_tiles(const CullData &d, const Grid &g, int ty, int &ka, int &kb) {
    if (!(d.T >= 0.f)) return false;
    const float y0 = (float)(ty * g.th), y1 = (float)(min(ty * g.th + g.th - 1, g.H - 1) + g.ext);
    float lo = __int_as_float(0x7f800000), hi = __int_as_float(0xff800000);
    if (d.yl >= y0 && d.yl <= y1) lo = __fsub_rn(d.mx, d.ex);
    if (d.yr >= y0 && d.yr <= y1) hi = __fadd_rn(d.mx, d.ex);
#pragma unroll
    for (int e = 0; e < 2; ++e) {
        const float dY = __fsub_rn(e == 0 ? y0 : y1, d.my);
        const float disc = __fsub_rn(d.aT, __fmul_rn(__fmul_rn(d.det, dY), dY));
        if (disc >= 0.f) {
            const float rt = __fsqrt_rn(disc);
            const float nm = -__fmul_rn(d.b, dY);
            const float xl = __fadd_rn(d.mx, __fmul_rn(__fsub_rn(nm, rt), d.ia));
            const float xr = __fadd_rn(d.mx, __fmul_rn(__fadd_rn(nm, rt), d.ia));
            lo = fminf(lo, xl);
            hi = fmaxf(hi, xr);
        }
    }
    if (!(lo <= hi)) return false;
    if (lo > (float)(g.W - 1 + g.ext) || hi < 0.f) return false;
    const float iw = __frcp_rn((float)g.tw);  // exact: the tile width is a power of two
    float t = __fmul_rn(__fadd_rn(lo, (float)(1 - g.ext)), iw);
    float u = __fmul_rn(hi, iw);
    t = fmaxf(t, -1.f);
    u = fminf(u, (float)(g.W / g.tw + 2));
    ka = (int)ceilf(t) - 1;
    kb = (int)floorf(u);
    return ka <= kb;
}

// Kept columns of row ty inside the box columns [x0, x1); returns their count (0 if none).
__device__ __forceinline__ int row_span_in_box(const CullData &d, const Grid &g, int ty, int x0, int x1, int &ka,
                                               int &kb) {
    if (!row_tiles(d, g, ty, ka, kb)) return 0;
    ka = max(ka, x0);
    kb = min(kb, x1 - 1);
    return kb >= ka ? kb - ka + 1 : 0;
}

__device__ __forceinline__ bool keep_tile(const CullData &d, const Grid &g, int tx, int ty) {
    int ka, kb;
    return row_tiles(d, g, ty, ka, kb) && tx >= ka && tx <= kb;
}

// Slot r of a box of width bw starting at (bx, by) is tile (bx + r mod bw, by + r div bw).  A warp
// walks slots lane, lane + 32, ...; SlotWalk keeps each lane's tile and steps it by 32 slots with a
// carry instead of dividing per slot.
struct SlotWalk {
    int tx, ty, bx, bw, dq, dr;
    __device__ __forceinline__ SlotWalk(int bx_, int by_, int bw_, int lane) : bx(bx_), bw(bw_) {
        ty = by_ + lane / bw_;
        tx = bx_ + lane % bw_;
        dq = 32 / bw_;
        dr = 32 % bw_;
    }
    __device__ __forceinline__ void step() {
        tx += dr;
        ty += dq;
        if (tx >= bx + bw) {
            tx -= bw;
            ty += 1;
        }
    }
};

__host__ __device__ inline Grid make_grid(const XprCamera &cam, const XprConfig &cfg) {
    Grid g;
    g.W = cam.width;
    g.H = cam.height;
    g.tw = cfg.tile_w;
    g.th = cfg.tile_h;
    g.Wt = tiles_x(cam, cfg);
    g.Ht = tiles_y(cam, cfg);
    g.ext = cfg.method == XPR_METHOD_3DGUT ? 1 : 0;
    return g;
}

// Tile box of primitive i clamped to the grid (all zero when its tile count is 0); returns its
// number of tiles (0 for an empty box).
__device__ __forceinline__ int box_of(const int4 *__restrict__ bbox, const int *__restrict__ tcount, int i,
                                      const Grid &g, int4 &bb) {
    bb = make_int4(0, 0, 0, 0);
    if (tcount[i] <= 0) return 0;
    bb = bbox[i];
    bb.x = max(bb.x, 0);  // never leave the tile grid, whatever the caller's boxes say
    bb.y = max(bb.y, 0);
    bb.z = min(bb.z, g.Wt);
    bb.w = min(bb.w, g.Ht);
    const int w = bb.z - bb.x, h = bb.w - bb.y;
    return (w > 0 && h > 0) ? w * h : 0;
}

// Rows of the 32 boxes of a warp (one per lane) are processed flattened over the lanes: with
// incl = inclusive prefix over lanes of the boxes' row counts, flattened row f belongs to the
// first lane whose incl exceeds f (a binary search by shuffles; incl is non-decreasing).
__device__ __forceinline__ int lane_of(int incl, int f) {
    int r = 0;
#pragma unroll
    for (int step = 16; step >= 1; step >>= 1)
        if (__shfl_sync(kFullMask, incl, r + step - 1) <= f) r += step;
    return min(r, 31);
}

__device__ __forceinline__ int warp_incl_scan(int x) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(kFullMask, x, o);
        if (lane >= o) x += y;
    }
    return x;
}

// Number of kept tiles of each lane's box bb (area = tiles in bb, 0 for none), with the tile rows
// of the warp's boxes spread over the lanes 32 at a time.  Every lane of the warp must call this.
__device__ __forceinline__ int count_kept_tiles(const CullData &d, const int4 bb, int area, const Grid &g) {
    const int lane = threadIdx.x & 31;
    const int h = area > 0 ? bb.w - bb.y : 0;
    const int incl = warp_incl_scan(h);
    const int rows = __shfl_sync(kFullMask, incl, 31);
    const int excl = incl - h;
    int cnt = 0;
    for (int f0 = 0; f0 < rows; f0 += 32) {
        const int f = f0 + lane;
        const int p = lane_of(incl, f);
        const CullData e = shfl_cull(d, p);
        const int ty = __shfl_sync(kFullMask, bb.y, p) + f - __shfl_sync(kFullMask, excl, p);
        const int x0 = __shfl_sync(kFullMask, bb.x, p), x1 = __shfl_sync(kFullMask, bb.z, p);
        int ka, kb;
        const int c = f < rows ? row_span_in_box(e, g, ty, x0, x1, ka, kb) : 0;
        // this lane's rows in this step are the lanes [excl - f0, incl - 1 - f0] (clipped to the step)
        const int s = warp_incl_scan(c);
        const int lo = max(excl - f0, 0), hi = min(incl - 1 - f0, 31);
        const int s_hi = __shfl_sync(kFullMask, s, max(hi, 0));
        const int s_lo = __shfl_sync(kFullMask, s, max(lo - 1, 0));
        if (h > 0 && hi >= 0 && lo <= 31 && lo <= hi) cnt += s_hi - (lo > 0 ? s_lo : 0);
    }
    return cnt;
}

}  // namespace xpr
