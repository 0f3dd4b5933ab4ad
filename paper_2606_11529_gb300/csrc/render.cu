// Shader stage (Sec. 2 Shader; Sec. 4.3; Algorithm 1; Listing 1 evaluate) and its adjoint.
//
// Forward (K4): one thread block per tile, one thread per pixel.  The tile's depth-sorted list is
// consumed in batches: every thread stages one entry's shading record into shared memory, then each
// pixel walks the batch front to back:
//   power = -(c00 dx^2 + 2 c01 dx dy + c11 dy^2)/2  (base-2 form, conic pre-scaled by log2 e)
//   skip if power > 0;  alpha = min(alpha_max, o 2^power2);  skip if alpha < alpha_t
//   stop if T (1 - alpha) < t_eps (that entry is not blended);  C += c alpha T;  T *= 1 - alpha
// A block stops loading batches as soon as every pixel has terminated (__syncthreads_and), which
// replaces the paper's fixed trip counts and per-bin batch boundaries with a dynamic exit.
//
// Backward (K5): the same blocks re-walk the list back to front from each pixel's n_contrib,
// recomputing T_i = T_{i+1} / (1 - alpha_i) and the colour behind, S (starting at T_final bg):
//   dL/dc_i = g alpha_i T_i,   dL/dalpha_i = g . (c_i T_i - S_i / (1 - alpha_i))
// then through alpha = o exp(power) (zero through the clamp) to o, mu_2D and the conic.  The 9
// per-pixel partial gradients of one entry are summed over the warp with shuffles, over the block
// in shared memory, and added to global memory with one set of atomics per (tile, entry).
#include "xpr_internal.cuh"

namespace xpr {
namespace {

constexpr unsigned kFull = 0xffffffffu;

struct Consts {
    int W, H, Wt;
    uint32_t n;  // primitive count: list entries >= n are ignored
    float at, amax, teps, bg0, bg1, bg2;
};

template <int TW, int TH>
__global__ void __launch_bounds__(TW *TH) render_fwd_kernel(const float *__restrict__ rec,
                                                            const uint32_t *__restrict__ vals,
                                                            const int2 *__restrict__ ranges, Consts k,
                                                            float *__restrict__ image, float *__restrict__ tfin,
                                                            int *__restrict__ ncon) {
    constexpr int NT = TW * TH;
    __shared__ float4 s_g[NT];  // mx, my, A, B
    __shared__ float4 s_c[NT];  // C, o, r, g
    __shared__ float s_b[NT];   // b
    const int tile = blockIdx.x;
    const int tx = tile % k.Wt, ty = tile / k.Wt;
    const int t = threadIdx.x;
    const int px = tx * TW + (t % TW), py = ty * TH + (t / TW);
    const bool inside = (px < k.W) && (py < k.H);
    const int2 rg = ranges[tile];
    const float fx = (float)px, fy = (float)py;
    float T = 1.f, cr = 0.f, cg = 0.f, cb = 0.f;
    int last = 0;
    bool done = !inside;
    for (int base = rg.x; base < rg.y; base += NT) {
        if (__syncthreads_and(done)) break;
        const int e = base + t;
        if (e < rg.y) {
            const uint32_t id = __ldg(vals + e);
            const Shade s = id < k.n ? load_shade(rec, id) : Shade{0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
            s_g[t] = make_float4(s.mx, s.my, s.A, s.B);
            s_c[t] = make_float4(s.C, s.o, s.r, s.g);
            s_b[t] = s.b;
        }
        __syncthreads();
        if (!done) {
            const int cnt = min(NT, rg.y - base);
            for (int j = 0; j < cnt; ++j) {
                const float4 g = s_g[j];
                const float4 c = s_c[j];
                const float dx = __fsub_rn(fx, g.x), dy = __fsub_rn(fy, g.y);
                const float p = eval_power2(g.z, g.w, c.x, dx, dy);
                if (p > 0.f) continue;
                const float og = __fmul_rn(c.y, ex2_approx(p));
                const float al = fminf(k.amax, og);
                if (al < k.at) continue;
                const float tt = __fmul_rn(T, __fsub_rn(1.f, al));
                if (tt < k.teps) {
                    done = true;
                    break;
                }
                const float w = al * T;
                cr = fmaf(c.z, w, cr);
                cg = fmaf(c.w, w, cg);
                cb = fmaf(s_b[j], w, cb);
                T = tt;
                last = base + j - rg.x + 1;
            }
        }
    }
    if (inside) {
        const int64_t pix = (int64_t)py * k.W + px, HW = (int64_t)k.W * k.H;
        image[pix] = fmaf(T, k.bg0, cr);
        image[HW + pix] = fmaf(T, k.bg1, cg);
        image[2 * HW + pix] = fmaf(T, k.bg2, cb);
        tfin[pix] = T;
        ncon[pix] = last;
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
    for (int k = 0; k < 4; ++k) {
        const float send = u16 ? v[k] : v[k + 4];
        const float keep = u16 ? v[k + 4] : v[k];
        b[k] = keep + __shfl_xor_sync(kFull, send, 16);
    }
    float c[2];
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        const float send = u8 ? b[k] : b[k + 2];
        const float keep = u8 ? b[k + 2] : b[k];
        c[k] = keep + __shfl_xor_sync(kFull, send, 8);
    }
    float d = (u4 ? c[1] : c[0]) + __shfl_xor_sync(kFull, u4 ? c[0] : c[1], 4);
    d += __shfl_xor_sync(kFull, d, 2);
    d += __shfl_xor_sync(kFull, d, 1);
    return d;
}

template <int TW, int TH>
__global__ void __launch_bounds__(TW *TH) render_bwd_kernel(const float *__restrict__ rec,
                                                            const uint32_t *__restrict__ vals,
                                                            const int2 *__restrict__ ranges, Consts k,
                                                            const float *__restrict__ tfin,
                                                            const int *__restrict__ ncon,
                                                            const float *__restrict__ dimg,
                                                            float *__restrict__ d_rec) {
    constexpr int NT = TW * TH;
    constexpr int NW = NT / 32;
    __shared__ float4 s_g[NT];
    __shared__ float4 s_c[NT];
    __shared__ float s_b[NT];
    __shared__ uint32_t s_id[NT];
    __shared__ float s_acc[9][NT];
    __shared__ int s_wmax[NW];
    const int tile = blockIdx.x;
    const int tx = tile % k.Wt, ty = tile / k.Wt;
    const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
    const int px = tx * TW + (t % TW), py = ty * TH + (t / TW);
    const bool inside = (px < k.W) && (py < k.H);
    const int2 rg = ranges[tile];
    const float fx = (float)px, fy = (float)py;
    const int64_t pix = (int64_t)py * k.W + px, HW = (int64_t)k.W * k.H;
    float T = 1.f, g0 = 0.f, g1 = 0.f, g2 = 0.f;
    int last = 0;
    if (inside) {
        T = tfin[pix];
        last = ncon[pix];
        g0 = dimg[pix];
        g1 = dimg[HW + pix];
        g2 = dimg[2 * HW + pix];
    }
    float S0 = T * k.bg0, S1 = T * k.bg1, S2 = T * k.bg2;
    const int wlast = __reduce_max_sync(kFull, last);
    if (lane == 0) s_wmax[wid] = wlast;
    __syncthreads();
    int bmax = 0;
#pragma unroll
    for (int w = 0; w < NW; ++w) bmax = max(bmax, s_wmax[w]);

    for (int end = rg.x + bmax; end > rg.x; end -= NT) {
        const int start = max(rg.x, end - NT);
        const int cnt = end - start;
        __syncthreads();
        if (t < cnt) {
            const uint32_t id = __ldg(vals + start + t);
            const Shade s = id < k.n ? load_shade(rec, id) : Shade{0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
            s_g[t] = make_float4(s.mx, s.my, s.A, s.B);
            s_c[t] = make_float4(s.C, s.o, s.r, s.g);
            s_b[t] = s.b;
            s_id[t] = id;
#pragma unroll
            for (int c = 0; c < 9; ++c) s_acc[c][t] = 0.f;
        }
        __syncthreads();
        for (int j = cnt - 1; j >= 0; --j) {
            const int pos = start + j - rg.x;
            if (pos >= wlast) continue;  // warp-uniform: no pixel of this warp reached the entry
            float v[9];
#pragma unroll
            for (int c = 0; c < 9; ++c) v[c] = 0.f;
            bool hit = false;
            if (pos < last) {
                const float4 g = s_g[j];
                const float4 c = s_c[j];
                const float dx = __fsub_rn(fx, g.x), dy = __fsub_rn(fy, g.y);
                const float p = eval_power2(g.z, g.w, c.x, dx, dy);
                if (p <= 0.f) {
                    const float G = ex2_approx(p);
                    const float og = __fmul_rn(c.y, G);
                    const float al = fminf(k.amax, og);
                    if (al >= k.at) {
                        hit = true;
                        const float cb = s_b[j];
                        const float inv = __frcp_rn(1.f - al);
                        const float Ti = T * inv;
                        const float w = al * Ti;
                        v[6] = g0 * w;
                        v[7] = g1 * w;
                        v[8] = g2 * w;
                        const float dal = g0 * (c.z * Ti - S0 * inv) + g1 * (c.w * Ti - S1 * inv) +
                                          g2 * (cb * Ti - S2 * inv);
                        S0 = fmaf(c.z, w, S0);
                        S1 = fmaf(c.w, w, S1);
                        S2 = fmaf(cb, w, S2);
                        T = Ti;
                        if (og < k.amax) {
                            const float dp = dal * al;  // dL/dpower (natural log units)
                            v[5] = dal * G;
                            v[0] = dp * fmaf(2.f * g.z, dx, g.w * dy);
                            v[1] = dp * fmaf(g.w, dx, 2.f * c.x * dy);
                            v[2] = dp * dx * dx;
                            v[3] = dp * dx * dy;
                            v[4] = dp * dy * dy;
                        }
                    }
                }
            }
            if (__any_sync(kFull, hit)) {
                // v[0..7]: transposed reduce-scatter (9 shuffles); afterwards lane l with l % 4 == 0
                // holds the warp total of value l / 4.  v[8]: plain butterfly (5 shuffles).
                const float s8 = warp_sum(v[8]);
                const float r7 = reduce_scatter8(v, lane);
                if ((lane & 3) == 0) atomicAdd(&s_acc[lane >> 2][j], r7);
                if (lane == 0) atomicAdd(&s_acc[8][j], s8);
            }
        }
        __syncthreads();
        if (t < cnt) {
            float a[9];
            bool any = false;
#pragma unroll
            for (int c = 0; c < 9; ++c) {
                a[c] = s_acc[c][t];
                any |= (a[c] != 0.f);
            }
            if (any && s_id[t] < k.n) {
                // record layout: [dmx, dmy, dc00, dc01] [dc11, do, dr, dg] [db, 0, 0, 0]; vector atomics
                float4 *d = reinterpret_cast<float4 *>(d_rec + (size_t)s_id[t] * XPR_REC_FLOATS);
                atomicAdd(d, make_float4(-kLn2 * a[0], -kLn2 * a[1], -0.5f * a[2], -a[3]));
                atomicAdd(d + 1, make_float4(-0.5f * a[4], a[5], a[6], a[7]));
                atomicAdd(reinterpret_cast<float *>(d + 2), a[8]);
            }
        }
    }
}

Consts make_consts(const XprCamera &cam, const XprConfig &cfg, int64_t n) {
    Consts k;
    k.n = (uint32_t)n;
    k.W = cam.width;
    k.H = cam.height;
    k.Wt = tiles_x(cam, cfg);
    k.at = cfg.alpha_thresh;
    k.amax = cfg.alpha_max;
    k.teps = cfg.t_eps;
    k.bg0 = cfg.bg[0];
    k.bg1 = cfg.bg[1];
    k.bg2 = cfg.bg[2];
    return k;
}

}  // namespace

#define XPR_TILE_DISPATCH(TWV, THV, CALL)                                                  \
    if (cfg.tile_w == 16 && cfg.tile_h == 16) { constexpr int TWV = 16, THV = 16; CALL; }  \
    else if (cfg.tile_w == 8 && cfg.tile_h == 8) { constexpr int TWV = 8, THV = 8; CALL; } \
    else if (cfg.tile_w == 16 && cfg.tile_h == 8) { constexpr int TWV = 16, THV = 8; CALL; } \
    else { constexpr int TWV = 8, THV = 16; CALL; }

int launch_render_fwd(const float *rec, int64_t n, const uint32_t *vals, const int32_t *ranges,
                      const XprCamera &cam, const XprConfig &cfg, float *image, float *t_final, int32_t *n_contrib,
                      cudaStream_t st) {
    const Consts k = make_consts(cam, cfg, n);
    const unsigned nt = (unsigned)(tiles_x(cam, cfg) * tiles_y(cam, cfg));
    const int2 *rg = reinterpret_cast<const int2 *>(ranges);
    XPR_TILE_DISPATCH(TW, TH, (render_fwd_kernel<TW, TH><<<nt, TW * TH, 0, st>>>(rec, vals, rg, k, image, t_final,
                                                                                   n_contrib)));
    XPR_LAUNCH_CHECK("render_fwd_kernel");
    return XPR_OK;
}

int launch_render_bwd(const float *rec, const uint32_t *vals, const int32_t *ranges, const XprCamera &cam,
                      const XprConfig &cfg, const float *t_final, const int32_t *n_contrib, const float *d_image,
                      float *d_rec, int64_t n, cudaStream_t st) {
    XPR_CUDA_TRY(cudaMemsetAsync(d_rec, 0, (size_t)n * XPR_REC_FLOATS * sizeof(float), st));
    const Consts k = make_consts(cam, cfg, n);
    const unsigned nt = (unsigned)(tiles_x(cam, cfg) * tiles_y(cam, cfg));
    const int2 *rg = reinterpret_cast<const int2 *>(ranges);
    XPR_TILE_DISPATCH(TW, TH, (render_bwd_kernel<TW, TH><<<nt, TW * TH, 0, st>>>(rec, vals, rg, k, t_final, n_contrib,
                                                                                   d_image, d_rec)));
    XPR_LAUNCH_CHECK("render_bwd_kernel");
    return XPR_OK;
}

}  // namespace xpr
