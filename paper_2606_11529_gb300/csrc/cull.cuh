// StopThePop tile cull of Listing 1 tile_cull, shared by the projection kernel (which counts the
// kept tiles of each primitive) and the emit kernel (which writes them).  Both must take identical
// decisions, so the decision is made in FP32 with one correctly rounded IEEE operation per step
// (explicit __f*_rn intrinsics, no contraction) on the stored float32 record values.
//
// The largest response o exp(-q/2), q = d^T conic d, d = mu_2D - p, over a tile is at mu_2D when
// mu_2D lies in the tile, else at the best point of the (at most two) tile edges facing mu_2D; on
// an edge the 1-D quadratic is minimised in closed form and clamped to the edge.  The pair is kept
// iff q/2 <= ln(o / alpha_t).  Tile bounds are inclusive pixel coordinates:
// x0 = tx w, x1 = min(tx w + w - 1, W - 1), same in y.
#pragma once

#include "xpr_internal.cuh"

namespace xpr {

struct CullData {
    float mx, my, c0, c1, c2, lt;
    float ic0, ic2;  // correctly rounded 1/c0 and 1/c2, computed once per primitive
};

__device__ __forceinline__ void cull_reciprocals(CullData &d) {
    d.ic0 = __frcp_rn(d.c0);
    d.ic2 = __frcp_rn(d.c2);
}

struct Grid {
    int W, H, tw, th, Wt, Ht;
};

constexpr unsigned kFullMask = 0xffffffffu;
constexpr int kSmallBox = 16;  // boxes with more tiles than this are walked by a whole warp

__device__ __forceinline__ float cull_quad_half(float c0, float c1, float c2, float dx, float dy) {
    float a = __fmul_rn(__fmul_rn(dx, dx), c0);
    float b = __fmul_rn(__fmul_rn(dx, dy), c1);
    b = __fadd_rn(b, b);
    float c = __fmul_rn(__fmul_rn(dy, dy), c2);
    return __fmul_rn(0.5f, __fadd_rn(__fadd_rn(a, b), c));
}

__device__ __forceinline__ bool tile_keep(const CullData &d, float x0, float y0, float x1, float y1) {
    const bool outx = (d.mx < x0) || (d.mx > x1);
    const bool outy = (d.my < y0) || (d.my > y1);
    if (!outx && !outy) return 0.f <= d.lt;
    float best = __int_as_float(0x7f800000);
    if (outx) {
        const float ex = d.mx < x0 ? x0 : x1;
        const float dx = __fsub_rn(d.mx, ex);
        float ys = __fadd_rn(d.my, __fmul_rn(__fmul_rn(d.c1, dx), d.ic2));
        ys = fminf(fmaxf(ys, y0), y1);
        const float dy = __fsub_rn(d.my, ys);
        best = fminf(best, cull_quad_half(d.c0, d.c1, d.c2, dx, dy));
    }
    if (outy) {
        const float ey = d.my < y0 ? y0 : y1;
        const float dy = __fsub_rn(d.my, ey);
        float xs = __fadd_rn(d.mx, __fmul_rn(__fmul_rn(d.c1, dy), d.ic0));
        xs = fminf(fmaxf(xs, x0), x1);
        const float dx = __fsub_rn(d.mx, xs);
        best = fminf(best, cull_quad_half(d.c0, d.c1, d.c2, dx, dy));
    }
    return best <= d.lt;
}

__device__ __forceinline__ bool keep_tile(const CullData &d, const Grid &g, int tx, int ty) {
    const float x0 = (float)(tx * g.tw), x1 = (float)min(tx * g.tw + g.tw - 1, g.W - 1);
    const float y0 = (float)(ty * g.th), y1 = (float)min(ty * g.th + g.th - 1, g.H - 1);
    return tile_keep(d, x0, y0, x1, y1);
}

__device__ __forceinline__ CullData load_cull(const float *__restrict__ rec, int64_t i) {
    const float4 *p = reinterpret_cast<const float4 *>(rec + (size_t)i * XPR_REC_FLOATS);
    const float4 a = __ldg(p), b = __ldg(p + 1), c = __ldg(p + 2);
    CullData d;
    d.mx = a.x;
    d.my = a.y;
    d.c0 = a.z;
    d.c1 = a.w;
    d.c2 = b.x;
    d.lt = c.z;
    cull_reciprocals(d);
    return d;
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
    return g;
}

// Number of kept tiles of each lane's box bb (area = tiles in bb, 0 for none).  Boxes of at most
// kSmallBox tiles are counted by their own lane; larger ones by the whole warp, one box at a time.
// Every lane of the warp must call this.
__device__ __forceinline__ int count_kept_tiles(const CullData &d, const int4 bb, int area, const Grid &g) {
    const int lane = threadIdx.x & 31;
    int cnt = 0;
    if (area > 0 && area <= kSmallBox) {
        for (int ty = bb.y; ty < bb.w; ++ty)
            for (int tx = bb.x; tx < bb.z; ++tx) cnt += keep_tile(d, g, tx, ty) ? 1 : 0;
    }
    unsigned big = __ballot_sync(kFullMask, area > kSmallBox);
    while (big) {
        const int src = __ffs(big) - 1;
        big &= big - 1;
        CullData e;
        e.mx = __shfl_sync(kFullMask, d.mx, src);
        e.my = __shfl_sync(kFullMask, d.my, src);
        e.c0 = __shfl_sync(kFullMask, d.c0, src);
        e.c1 = __shfl_sync(kFullMask, d.c1, src);
        e.c2 = __shfl_sync(kFullMask, d.c2, src);
        e.lt = __shfl_sync(kFullMask, d.lt, src);
        e.ic0 = __shfl_sync(kFullMask, d.ic0, src);
        e.ic2 = __shfl_sync(kFullMask, d.ic2, src);
        const int areab = __shfl_sync(kFullMask, area, src);
        const int bx = __shfl_sync(kFullMask, bb.x, src), by = __shfl_sync(kFullMask, bb.y, src);
        const int bw = __shfl_sync(kFullMask, bb.z, src) - bx;
        SlotWalk sw(bx, by, bw, lane);
        int c = 0;
        for (int r0 = 0; r0 < areab; r0 += 32) {
            const bool keep = r0 + lane < areab && keep_tile(e, g, sw.tx, sw.ty);
            c += __popc(__ballot_sync(kFullMask, keep));
            sw.step();
        }
        if (lane == src) cnt = c;
    }
    return cnt;
}

}  // namespace xpr
