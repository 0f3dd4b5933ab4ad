// Shader stage (Sec. 2 Shader; Sec. 4.3; Algorithm 1; Listing 1 evaluate) and its adjoint.
//
// Forward (K4): one thread block per tile; each thread owns PX pixels of one pixel column of the
// tile (4 in the forward, 8 in the adjoint on 16x16 tiles), so every shared-memory read of a list
// entry, the column factors of the power and every warp reduction of the adjoint serve PX pixels.
// The tile's depth-sorted list is consumed in batches of `batch` entries staged in shared memory,
// then each pixel walks the batch front to back:
//   power = -(c00 dx^2 + 2 c01 dx dy + c11 dy^2)/2  (base-2 form, conic pre-scaled by log2 e)
//   skip if power > 0;  alpha = min(alpha_max, o 2^power2);  skip if alpha < alpha_t
//   stop if T (1 - alpha) < t_eps (that entry is not blended);  C += c alpha T;  T *= 1 - alpha
// Every pixel evaluates every entry with no early exit: the gates are predicates (the forward's
// blend a predicated block, the adjoint's updates selects that add zeros for a pixel the entry
// does not reach), so a warp runs one straight path per entry.
// A block stops loading batches as soon as every pixel has terminated (__syncthreads_and), which
// replaces the paper's fixed trip counts and per-bin batch boundaries with a dynamic exit.
//
// Backward (K5): the same blocks re-walk the list back to front from each pixel's n_contrib,
// recomputing T_i = T_{i+1} / (1 - alpha_i) and the colour behind, S (starting at T_final bg):
//   dL/dc_i = g alpha_i T_i,   dL/dalpha_i = g . (c_i T_i - S_i / (1 - alpha_i))
// S enters only through g . S, so each pixel carries that scalar, B (B += (g . c_i) alpha_i T_i).
// then through alpha = o exp(power) (zero through the clamp) to o, mu_2D and the conic.  The
// mean's partials d power / d mu_2D = -(2A dx + B dy, B dx + 2C dy) are linear in (dx, dy) with
// per-entry factors, so a pixel accumulates only dp dx and dp dy (with dp dx^2, dp dx dy, dp dy^2
// for the conic) and the factors are applied once per (tile, entry).  The 9 per-pixel partials
// of one entry are summed over the thread's pixels, over the warp with shuffles, over the block
// in shared memory, and added to global memory with one set of vector atomics per (tile, entry).
//
// Views: tile gt of a multi-view launch is tile gt mod T of view gt div T (T tiles per view, all
// views of one size); images are [views, 3, H, W].  Scheduling: one block per tile, or a
// persistent grid whose blocks take tiles from a work list (tiles by descending list length,
// the paper's trip-count binning made dynamic) through an atomic counter.
#include "xpr_internal.cuh"

namespace xpr {
namespace {

constexpr unsigned kFull = 0xffffffffu;
// Pixels per thread: (x, y + q h/PX), q = 0..PX-1, with PX = min(cap, tile pixels / 32) so that a
// tile's block is always whole warps (warp-wide shuffles and votes need all 32 lanes).  The caps
// of the forward (4) and the adjoint (8: one warp per 16x16 tile, each warp reduction serving 8
// pixels) are compile-time constants.
#ifndef XPR_FWD_PX
#define XPR_FWD_PX 4
#endif
#ifndef XPR_BWD_PX
#define XPR_BWD_PX 8
#endif
template <int TW, int TH, int CAP>
__host__ __device__ constexpr int px_cap() {
    return (TW * TH) / 32 >= CAP ? CAP : (TW * TH) / 32;
}
template <int TW, int TH>
__host__ __device__ constexpr int fwd_px() {
    return px_cap<TW, TH, XPR_FWD_PX>();
}
template <int TW, int TH>
__host__ __device__ constexpr int bwd_px() {
    return px_cap<TW, TH, XPR_BWD_PX>();
}
constexpr int kMaxBatch = 256;  // largest shared-memory batch (entries)
// The adjoint stages at most kBwdBatch entries: its 9 accumulator rows make a block's shared
// memory grow 2.3x faster with the batch than the forward's, and at 256 entries shared memory
// alone held an SM to 11 blocks.
constexpr int kBwdBatch = 128;

struct Consts {
    int W, H, Wt, T;  // image size, tiles per row, tiles per view
    uint32_t n;       // number of records: list entries >= n are ignored
    int batch;        // entries staged per batch, 1 .. kMaxBatch
    float at, amax, teps, bg0, bg1, bg2;
    ItemTable it;     // multi-scene launch: per-item grids (it.count 0: uniform views)
};

// Where global tile gt lies: its item (or view), tile index within it, the item's image size and
// tiles per row, and its first pixel in the per-pixel buffers.
struct TileLoc {
    int v, tile, W, H, Wt;
    int64_t pix0;
};

__device__ __forceinline__ TileLoc locate(int gt, const Consts &k) {
    TileLoc l;
    if (k.it.count > 0) {
        l.v = item_of_tile(k.it, gt);
        l.tile = (int)(gt - k.it.tile0[l.v]);
        l.W = k.it.W[l.v];
        l.H = k.it.H[l.v];
        l.Wt = k.it.Wt[l.v];
        l.pix0 = k.it.pix0[l.v];
    } else {
        l.v = gt / k.T;
        l.tile = gt - l.v * k.T;
        l.W = k.W;
        l.H = k.H;
        l.Wt = k.Wt;
        l.pix0 = (int64_t)l.v * k.W * k.H;
    }
    return l;
}

struct Work {  // persistent scheduling: tiles list[0 .. count) taken through *counter
    const int *list;
    int *counter;
    int count;
};

__device__ __forceinline__ void stage(const float *__restrict__ rec, const uint32_t *__restrict__ vals, int e,
                                      uint32_t n, float4 *s_g, float4 *s_c, float *s_b, uint32_t *s_id, int slot) {
    const uint32_t id = __ldg(vals + e);
    const Shade s = id < n ? load_shade(rec, id) : Shade{0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    s_g[slot] = make_float4(s.mx, s.my, s.A, s.B);
    s_c[slot] = make_float4(s.C, s.o, s.r, s.g);
    s_b[slot] = s.b;
    if (s_id) s_id[slot] = id;
}

struct PixelFwd {
    float fy, T, r, g, b;
    int last;
    bool done;
};

// Blends entry (g, c, cb) at list position pos into pixel P (front to back).  No early exit: the
// gates are predicates and the blend a predicated block.  2^p needs no guard: for the
// positive-definite conic of a kept record p <= 0 up to rounding, and a non-finite value could
// only reach alpha, which the p <= 0 gate then discards.
__device__ __forceinline__ void blend(PixelFwd &P, const ColTerms &ct, const float4 &g, const float4 &c, float cb,
                                      int pos, const Consts &k) {
    const float dy = __fsub_rn(P.fy, g.y);
    const float p = eval_power2(ct, c.x, dy);
    const float og = __fmul_rn(c.y, ex2_approx(p));
    const float al = fminf(k.amax, og);
    const bool live = !P.done && p <= 0.f && al >= k.at;
    const float tt = __fmul_rn(P.T, __fsub_rn(1.f, al));
    const bool stop = live && tt < k.teps;
    if (live && !stop) {
        const float w = al * P.T;
        P.r = fmaf(c.z, w, P.r);
        P.g = fmaf(c.w, w, P.g);
        P.b = fmaf(cb, w, P.b);
        P.T = tt;
        P.last = pos + 1;
    }
    P.done = P.done || stop;
}

template <int TW, int TH>
__device__ __forceinline__ void fwd_tile(int gt, const float *__restrict__ rec, const uint32_t *__restrict__ vals,
                                         const int2 *__restrict__ ranges, const Consts &k, float *__restrict__ image,
                                         float *__restrict__ tfin, int *__restrict__ ncon, float4 *s_g, float4 *s_c,
                                         float *s_b) {
    constexpr int kPX = fwd_px<TW, TH>();
    constexpr int NT = TW * TH / kPX;
    constexpr int RS = TH / kPX;  // rows between a thread's pixels
    static_assert(NT % 32 == 0, "a tile's block must be whole warps");
    const TileLoc L = locate(gt, k);
    const int tx = L.tile % L.Wt, ty = L.tile / L.Wt;
    const int t = threadIdx.x;
    const int px = tx * TW + t % TW, py = ty * TH + t / TW;
    const int2 rg = ranges[gt];
    const float fx = (float)px;
    PixelFwd P[kPX];
    bool in[kPX];
    bool all_done = true;
#pragma unroll
    for (int q = 0; q < kPX; ++q) {
        in[q] = px < L.W && py + q * RS < L.H;
        P[q] = PixelFwd{(float)(py + q * RS), 1.f, 0.f, 0.f, 0.f, 0, !in[q]};
        all_done &= P[q].done;
    }
    for (int base = rg.x; base < rg.y; base += k.batch) {
        if (__syncthreads_and(all_done)) break;
        const int cnt = min(k.batch, rg.y - base);
        for (int e = t; e < cnt; e += NT) stage(rec, vals, base + e, k.n, s_g, s_c, s_b, nullptr, e);
        __syncthreads();
        if (!all_done) {
            for (int j = 0; j < cnt; ++j) {
                const float4 g = s_g[j];
                const float4 c = s_c[j];
                const float cb = s_b[j];
                const float dx = __fsub_rn(fx, g.x);
                const ColTerms ct = column_terms(g.z, g.w, dx);
                const int pos = base + j - rg.x;
                all_done = true;
#pragma unroll
                for (int q = 0; q < kPX; ++q) {
                    blend(P[q], ct, g, c, cb, pos, k);
                    all_done &= P[q].done;
                }
                if (all_done) break;
            }
        }
    }
    const int64_t HW = (int64_t)L.W * L.H;
    float *img = image + 3 * L.pix0;
#pragma unroll
    for (int q = 0; q < kPX; ++q) {
        if (!in[q]) continue;
        const int64_t pix = (int64_t)(py + q * RS) * L.W + px;
        img[pix] = fmaf(P[q].T, k.bg0, P[q].r);
        img[HW + pix] = fmaf(P[q].T, k.bg1, P[q].g);
        img[2 * HW + pix] = fmaf(P[q].T, k.bg2, P[q].b);
        tfin[L.pix0 + pix] = P[q].T;
        ncon[L.pix0 + pix] = P[q].last;
    }
}

template <int TW, int TH>
__global__ void __launch_bounds__(TW *TH / fwd_px<TW, TH>()) render_fwd_kernel(const float *__restrict__ rec,
                                                                  const uint32_t *__restrict__ vals,
                                                                  const int2 *__restrict__ ranges, Consts k,
                                                                  float *__restrict__ image,
                                                                  float *__restrict__ tfin, int *__restrict__ ncon,
                                                                  Work w) {
    grid_dep_wait();
    __shared__ float4 s_g[kMaxBatch];  // mx, my, A, B
    __shared__ float4 s_c[kMaxBatch];  // C, o, r, g
    __shared__ float s_b[kMaxBatch];   // b
    if (w.list == nullptr) {
        fwd_tile<TW, TH>(blockIdx.x, rec, vals, ranges, k, image, tfin, ncon, s_g, s_c, s_b);
        return;
    }
    __shared__ int s_item;
    for (;;) {
        if (threadIdx.x == 0) s_item = atomicAdd(w.counter, 1);
        __syncthreads();
        const int item = s_item;
        __syncthreads();
        if (item >= w.count) break;
        fwd_tile<TW, TH>(w.list[item], rec, vals, ranges, k, image, tfin, ncon, s_g, s_c, s_b);
    }
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    return v;
}

// Sum 8 per-lane values over the warp with 9 shuffles instead of 40: at each of the first three
// steps a lane keeps the half of its values selected by one bit of its lane index and sends the
// other half to its partner, so after xor 16, 8, 4 lane l holds value (l >> 2) summed over the 8
// lanes sharing bits 1..0; two more xor steps finish the sum.  Returns value (lane >> 2).
__device__ __forceinline__ float reduce_scatter8(const float *v, int lane) {
    const bool u16 = lane & 16, u8 = lane & 8, u4 = lane & 4;
    float b[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const float send = u16 ? v[q] : v[q + 4];
        const float keep = u16 ? v[q + 4] : v[q];
        b[q] = keep + __shfl_xor_sync(kFull, send, 16);
    }
    float c[2];
#pragma unroll
    for (int q = 0; q < 2; ++q) {
        const float send = u8 ? b[q] : b[q + 2];
        const float keep = u8 ? b[q + 2] : b[q];
        c[q] = keep + __shfl_xor_sync(kFull, send, 8);
    }
    float d = (u4 ? c[1] : c[0]) + __shfl_xor_sync(kFull, u4 ? c[0] : c[1], 4);
    d += __shfl_xor_sync(kFull, d, 2);
    d += __shfl_xor_sync(kFull, d, 1);
    return d;
}

struct PixelBwd {
    float fy, T, g0, g1, g2, B;  // B = g . (colour behind the current entry)
    int last;
};

// Adds pixel P's partial gradients for the entry at list position pos (back to front) into v[9]:
// v = [dp dx, dp dy, dp dx^2, dp dx dy, dp dy^2, dL/do, dL/dr, dL/dg, dL/db]; the conic factors of
// d power / d mu_2D (2A dx + B dy, B dx + 2C dy in the base-2 form) are applied at the flush.
// Branch-free: a pixel the entry does not reach adds zeros and keeps its state (selects; a
// predicated block measured slower here).  2^min(p, 0) keeps G finite for the products with
// the selected zeros.
__device__ __forceinline__ bool adjoint(PixelBwd &P, float dx, const ColTerms &ct, const float4 &g, const float4 &c,
                                        float cb, int pos, const Consts &k, float *v) {
    const float dy = __fsub_rn(P.fy, g.y);
    const float p = eval_power2(ct, c.x, dy);
    const float G = ex2_approx(fminf(p, 0.f));
    const float og = __fmul_rn(c.y, G);
    const float al = fminf(k.amax, og);
    const bool live = pos < P.last && p <= 0.f && al >= k.at;
    const float inv = rcp_approx(1.f - al);
    const float Ti = P.T * inv;
    const float w = live ? al * Ti : 0.f;
    v[6] = fmaf(P.g0, w, v[6]);
    v[7] = fmaf(P.g1, w, v[7]);
    v[8] = fmaf(P.g2, w, v[8]);
    const float gc = fmaf(P.g0, c.z, fmaf(P.g1, c.w, P.g2 * cb));
    const float dal = (live && og < k.amax) ? fmaf(gc, Ti, -P.B * inv) : 0.f;
    P.B = fmaf(gc, w, P.B);
    P.T = live ? Ti : P.T;
    const float dp = dal * al;  // dL/dpower (natural log units)
    v[5] = fmaf(dal, G, v[5]);
    const float dpx = dp * dx, dpy = dp * dy;
    v[0] += dpx;
    v[1] += dpy;
    v[2] = fmaf(dpx, dx, v[2]);
    v[3] = fmaf(dpx, dy, v[3]);
    v[4] = fmaf(dpy, dy, v[4]);
    return live;
}

__device__ __forceinline__ PixelBwd load_pixel_bwd(bool inside, float fy, int64_t pix, int64_t HW,
                                                   const float *__restrict__ tfin, const int *__restrict__ ncon,
                                                   const float *__restrict__ dimg, const Consts &k) {
    PixelBwd P = {fy, 1.f, 0.f, 0.f, 0.f, 0.f, 0};
    if (inside) {
        P.T = tfin[pix];
        P.last = ncon[pix];
        P.g0 = dimg[pix];
        P.g1 = dimg[HW + pix];
        P.g2 = dimg[2 * HW + pix];
    }
    P.B = P.T * fmaf(P.g0, k.bg0, fmaf(P.g1, k.bg1, P.g2 * k.bg2));
    return P;
}

template <int TW, int TH>
__device__ __forceinline__ void bwd_tile(int gt, const float *__restrict__ rec, const uint32_t *__restrict__ vals,
                                         const int2 *__restrict__ ranges, const Consts &k,
                                         const float *__restrict__ tfin, const int *__restrict__ ncon,
                                         const float *__restrict__ dimg, float *__restrict__ d_rec, float4 *s_g,
                                         float4 *s_c, float *s_b, uint32_t *s_id, float (*s_acc)[kBwdBatch + 1],
                                         int *s_wmax) {
    constexpr int kPX = bwd_px<TW, TH>();
    constexpr int NT = TW * TH / kPX;
    constexpr int NW = NT / 32;
    constexpr int RS = TH / kPX;
    static_assert(NT % 32 == 0, "a tile's block must be whole warps");
    const TileLoc L = locate(gt, k);
    const int tx = L.tile % L.Wt, ty = L.tile / L.Wt;
    const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
    const int px = tx * TW + t % TW, py = ty * TH + t / TW;
    const int2 rg = ranges[gt];
    const float fx = (float)px;
    const int64_t HW = (int64_t)L.W * L.H;
    const float *tf = tfin + L.pix0;
    const int *nc = ncon + L.pix0;
    const float *di = dimg + 3 * L.pix0;
    PixelBwd P[kPX];
    int mylast = 0;
#pragma unroll
    for (int q = 0; q < kPX; ++q) {
        const int y = py + q * RS;
        const bool in = px < L.W && y < L.H;
        P[q] = load_pixel_bwd(in, (float)y, (int64_t)y * L.W + px, HW, tf, nc, di, k);
        mylast = max(mylast, P[q].last);
    }
    const int wlast = __reduce_max_sync(kFull, mylast);
    if (lane == 0) s_wmax[wid] = wlast;
    __syncthreads();
    int bmax = 0;
#pragma unroll
    for (int w = 0; w < NW; ++w) bmax = max(bmax, s_wmax[w]);

    for (int end = rg.x + bmax; end > rg.x; end -= k.batch) {
        const int start = max(rg.x, end - k.batch);
        const int cnt = end - start;
        __syncthreads();
        for (int e = t; e < cnt; e += NT) {
            stage(rec, vals, start + e, k.n, s_g, s_c, s_b, s_id, e);
#pragma unroll
            for (int c = 0; c < 9; ++c) s_acc[c][e] = 0.f;
        }
        __syncthreads();
        for (int j = cnt - 1; j >= 0; --j) {
            const int pos = start + j - rg.x;
            if (pos >= wlast) continue;  // warp-uniform: no pixel of this warp reached the entry
            float vv[9];
#pragma unroll
            for (int c = 0; c < 9; ++c) vv[c] = 0.f;
            const float4 g = s_g[j];
            const float4 c = s_c[j];
            const float cb = s_b[j];
            const float dx = __fsub_rn(fx, g.x);
            const ColTerms ct = column_terms(g.z, g.w, dx);
            bool hit = false;
#pragma unroll
            for (int q = 0; q < kPX; ++q) hit |= adjoint(P[q], dx, ct, g, c, cb, pos, k, vv);
            if (__any_sync(kFull, hit)) {
                // vv[0..7]: transposed reduce-scatter (9 shuffles); afterwards lane l with l % 4 == 0
                // holds the warp total of value l / 4.  vv[8]: plain butterfly (5 shuffles).
                const float s8 = warp_sum(vv[8]);
                const float r7 = reduce_scatter8(vv, lane);
                if (NW == 1) {  // one warp per tile: each slot is written once
                    if ((lane & 3) == 0) s_acc[lane >> 2][j] = r7;
                    if (lane == 0) s_acc[8][j] = s8;
                } else {
                    if ((lane & 3) == 0) atomicAdd(&s_acc[lane >> 2][j], r7);
                    if (lane == 0) atomicAdd(&s_acc[8][j], s8);
                }
            }
        }
        __syncthreads();
        for (int e = t; e < cnt; e += NT) {
            float a[9];
            bool any = false;
#pragma unroll
            for (int c = 0; c < 9; ++c) {
                a[c] = s_acc[c][e];
                any |= (a[c] != 0.f);
            }
            if (any && s_id[e] < k.n) {
                // record layout: [dmx, dmy, dc00, dc01] [dc11, do, dr, dg] [db, 0, 0, 0]; vector atomics
                float4 *d = reinterpret_cast<float4 *>(d_rec + (size_t)s_id[e] * XPR_REC_FLOATS);
                const float A2 = 2.f * s_g[e].z, Bc = s_g[e].w, C2 = 2.f * s_c[e].x;
                const float qx = fmaf(A2, a[0], Bc * a[1]), qy = fmaf(Bc, a[0], C2 * a[1]);
                atomicAdd(d, make_float4(-kLn2 * qx, -kLn2 * qy, -0.5f * a[2], -a[3]));
                atomicAdd(d + 1, make_float4(-0.5f * a[4], a[5], a[6], a[7]));
                atomicAdd(reinterpret_cast<float *>(d + 2), a[8]);
            }
        }
    }
}

template <int TW, int TH>
__global__ void __launch_bounds__(TW *TH / bwd_px<TW, TH>()) render_bwd_kernel(const float *__restrict__ rec,
                                                                  const uint32_t *__restrict__ vals,
                                                                  const int2 *__restrict__ ranges, Consts k,
                                                                  const float *__restrict__ tfin,
                                                                  const int *__restrict__ ncon,
                                                                  const float *__restrict__ dimg,
                                                                  float *__restrict__ d_rec, Work w) {
    grid_dep_wait();
    __shared__ float4 s_g[kBwdBatch];
    __shared__ float4 s_c[kBwdBatch];
    __shared__ float s_b[kBwdBatch];
    __shared__ uint32_t s_id[kBwdBatch];
    // rows padded by one float: the 8 lanes adding one entry's values hit 8 different banks
    __shared__ float s_acc[9][kBwdBatch + 1];
    __shared__ int s_wmax[8];
    if (w.list == nullptr) {
        bwd_tile<TW, TH>(blockIdx.x, rec, vals, ranges, k, tfin, ncon, dimg, d_rec, s_g, s_c, s_b, s_id, s_acc,
                         s_wmax);
        return;
    }
    __shared__ int s_item;
    for (;;) {
        __syncthreads();  // the previous tile's last reads of shared memory are done
        if (threadIdx.x == 0) s_item = atomicAdd(w.counter, 1);
        __syncthreads();
        const int item = s_item;
        if (item >= w.count) break;
        bwd_tile<TW, TH>(w.list[item], rec, vals, ranges, k, tfin, ncon, dimg, d_rec, s_g, s_c, s_b, s_id, s_acc,
                         s_wmax);
    }
}

Consts make_consts(const XprCamera &cam, const XprConfig &cfg, int64_t n) {
    Consts k;
    k.n = (uint32_t)n;
    k.W = cam.width;
    k.H = cam.height;
    k.Wt = tiles_x(cam, cfg);
    k.T = tiles_x(cam, cfg) * tiles_y(cam, cfg);
    k.batch = cfg.batch_depth > 0 ? min(cfg.batch_depth, kMaxBatch) : kMaxBatch;
    k.at = cfg.alpha_thresh;
    k.amax = cfg.alpha_max;
    k.teps = cfg.t_eps;
    k.bg0 = cfg.bg[0];
    k.bg1 = cfg.bg[1];
    k.bg2 = cfg.bg[2];
    k.it.count = 0;
    return k;
}

template <typename KernelT>
int persistent_grid(KernelT kernel, int threads, int items) {
    int dev = 0, sms = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return items;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return items;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, 0) != cudaSuccess || per_sm < 1)
        per_sm = 1;
    return max(1, min(items, sms * per_sm));
}

}  // namespace

#define XPR_TILE_DISPATCH(TWV, THV, ...)                                                         \
    if (cfg.tile_w == 16 && cfg.tile_h == 16) { constexpr int TWV = 16, THV = 16; __VA_ARGS__; }  \
    else if (cfg.tile_w == 8 && cfg.tile_h == 8) { constexpr int TWV = 8, THV = 8; __VA_ARGS__; } \
    else if (cfg.tile_w == 16 && cfg.tile_h == 8) { constexpr int TWV = 16, THV = 8; __VA_ARGS__; } \
    else { constexpr int TWV = 8, THV = 16; __VA_ARGS__; }

// worklist/counter NULL: one block per tile over n_views * T tiles.  Otherwise a persistent grid
// walks worklist[0 .. n_views * T); *counter is zeroed here.
int launch_render_fwd_views(const float *rec, int64_t n, const uint32_t *vals, const int32_t *ranges, int n_views,
                            const XprCamera &cam, const XprConfig &cfg, float *image, float *t_final,
                            int32_t *n_contrib, const int32_t *worklist, int32_t *counter, cudaStream_t st) {
    const Consts k = make_consts(cam, cfg, n);
    const int items = n_views * k.T;
    if (items == 0) return XPR_OK;
    const int2 *rg = reinterpret_cast<const int2 *>(ranges);
    Work w = {worklist, counter, items};
    if (worklist) XPR_CUDA_TRY(cudaMemsetAsync(counter, 0, sizeof(int32_t), st));
    XPR_TILE_DISPATCH(TW, TH, {
        const int threads = TW * TH / fwd_px<TW, TH>();
        const int grid = worklist ? persistent_grid(render_fwd_kernel<TW, TH>, threads, items) : items;
        XPR_CUDA_TRY(launch_dependent(render_fwd_kernel<TW, TH>, dim3(grid), dim3(threads), 0, st, rec, vals, rg, k,
                                      image, t_final, n_contrib, w));
    });
    XPR_LAUNCH_CHECK("render_fwd_kernel");
    return XPR_OK;
}

int launch_render_bwd_views(const float *rec, const uint32_t *vals, const int32_t *ranges, int n_views,
                            const XprCamera &cam, const XprConfig &cfg, const float *t_final,
                            const int32_t *n_contrib, const float *d_image, float *d_rec, int64_t n,
                            const int32_t *worklist, int32_t *counter, cudaStream_t st) {
    XPR_CUDA_TRY(cudaMemsetAsync(d_rec, 0, (size_t)n * XPR_REC_FLOATS * sizeof(float), st));
    Consts k = make_consts(cam, cfg, n);
    k.batch = min(k.batch, kBwdBatch);
    const int items = n_views * k.T;
    if (items == 0) return XPR_OK;
    const int2 *rg = reinterpret_cast<const int2 *>(ranges);
    Work w = {worklist, counter, items};
    if (worklist) XPR_CUDA_TRY(cudaMemsetAsync(counter, 0, sizeof(int32_t), st));
    XPR_TILE_DISPATCH(TW, TH, {
        const int threads = TW * TH / bwd_px<TW, TH>();
        const int grid = worklist ? persistent_grid(render_bwd_kernel<TW, TH>, threads, items) : items;
        XPR_CUDA_TRY(launch_dependent(render_bwd_kernel<TW, TH>, dim3(grid), dim3(threads), 0, st, rec, vals, rg, k,
                                      t_final, n_contrib, d_image, d_rec, w));
    });
    XPR_LAUNCH_CHECK("render_bwd_kernel");
    return XPR_OK;
}

// Multi-scene launches: the tiles of every item in one grid (a persistent one over worklist when
// given); records are the items' concatenated blocks (n_rec in all).
int launch_render_fwd_items(const float *rec, int64_t n_rec, const uint32_t *vals, const int32_t *ranges,
                            const ItemTable &it, const XprConfig &cfg, float *image, float *t_final,
                            int32_t *n_contrib, const int32_t *worklist, int32_t *counter, cudaStream_t st) {
    XprCamera dummy = {};
    dummy.width = it.W[0];
    dummy.height = it.H[0];
    Consts k = make_consts(dummy, cfg, n_rec);
    k.it = it;
    const int64_t items = it.tile0[it.count];
    if (items == 0) return XPR_OK;
    if (items > 0x7fffffffLL) return fail(XPR_ERR_INVALID, "xpr_render_fwd_items: too many tiles");
    const int2 *rg = reinterpret_cast<const int2 *>(ranges);
    Work w = {worklist, counter, (int)items};
    if (worklist) XPR_CUDA_TRY(cudaMemsetAsync(counter, 0, sizeof(int32_t), st));
    XPR_TILE_DISPATCH(TW, TH, {
        const int threads = TW * TH / fwd_px<TW, TH>();
        const int grid = worklist ? persistent_grid(render_fwd_kernel<TW, TH>, threads, (int)items) : (int)items;
        XPR_CUDA_TRY(launch_dependent(render_fwd_kernel<TW, TH>, dim3(grid), dim3(threads), 0, st, rec, vals, rg, k,
                                      image, t_final, n_contrib, w));
    });
    XPR_LAUNCH_CHECK("render_fwd_kernel");
    return XPR_OK;
}

int launch_render_bwd_items(const float *rec, int64_t n_rec, const uint32_t *vals, const int32_t *ranges,
                            const ItemTable &it, const XprConfig &cfg, const float *t_final,
                            const int32_t *n_contrib, const float *d_image, float *d_rec, const int32_t *worklist,
                            int32_t *counter, cudaStream_t st) {
    XPR_CUDA_TRY(cudaMemsetAsync(d_rec, 0, (size_t)n_rec * XPR_REC_FLOATS * sizeof(float), st));
    XprCamera dummy = {};
    dummy.width = it.W[0];
    dummy.height = it.H[0];
    Consts k = make_consts(dummy, cfg, n_rec);
    k.it = it;
    k.batch = min(k.batch, kBwdBatch);
    const int64_t items = it.tile0[it.count];
    if (items == 0) return XPR_OK;
    if (items > 0x7fffffffLL) return fail(XPR_ERR_INVALID, "xpr_render_bwd_items: too many tiles");
    const int2 *rg = reinterpret_cast<const int2 *>(ranges);
    Work w = {worklist, counter, (int)items};
    if (worklist) XPR_CUDA_TRY(cudaMemsetAsync(counter, 0, sizeof(int32_t), st));
    XPR_TILE_DISPATCH(TW, TH, {
        const int threads = TW * TH / bwd_px<TW, TH>();
        const int grid = worklist ? persistent_grid(render_bwd_kernel<TW, TH>, threads, (int)items) : (int)items;
        XPR_CUDA_TRY(launch_dependent(render_bwd_kernel<TW, TH>, dim3(grid), dim3(threads), 0, st, rec, vals, rg, k,
                                      t_final, n_contrib, d_image, d_rec, w));
    });
    XPR_LAUNCH_CHECK("render_bwd_kernel");
    return XPR_OK;
}

int launch_render_fwd(const float *rec, int64_t n, const uint32_t *vals, const int32_t *ranges,
                      const XprCamera &cam, const XprConfig &cfg, float *image, float *t_final, int32_t *n_contrib,
                      cudaStream_t st) {
    return launch_render_fwd_views(rec, n, vals, ranges, 1, cam, cfg, image, t_final, n_contrib, nullptr, nullptr, st);
}

int launch_render_bwd(const float *rec, const uint32_t *vals, const int32_t *ranges, const XprCamera &cam,
                      const XprConfig &cfg, const float *t_final, const int32_t *n_contrib, const float *d_image,
                      float *d_rec, int64_t n, cudaStream_t st) {
    return launch_render_bwd_views(rec, vals, ranges, 1, cam, cfg, t_final, n_contrib, d_image, d_rec, n, nullptr,
                                   nullptr, st);
}

}  // namespace xpr
