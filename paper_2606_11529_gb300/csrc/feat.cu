// Rendered features (the "rendered feature" class of the design space: depth, semantics): the 3DGS
// compositing loop with extra channels.  Channel c of a pixel is sum_i f_ic alpha_i T_i over the
// colour's contributors and weights (zero background); the channels are the caller's per-primitive
// feature rows feat[n, n_feat] and, with with_depth, one more channel whose values are the records'
// depths (camera z).  One block per tile; the colour arithmetic is that of render.cu, so the image
// equals xpr_render_fwd's bit for bit.
//
// Adjoint: the compositing adjoint over all channels, dL/dalpha_i = sum_ch g_ch (v_ich T_i -
// S_ich / (1 - alpha_i)) with S the suffix sums recomputed back to front (colour channels start at
// T_final bg, feature channels at 0); S enters only through B = sum_ch g_ch S_ch, so each pixel
// carries that scalar (B += (sum_ch g_ch v_ich) alpha_i T_i).  Then through alpha as the colour-only
// adjoint; per entry the
// 9 record partials and the NF feature partials are summed over the warp (32-lane reduce-scatter)
// and the block, then added with atomics: d_rec in the record layout with the depth channel's
// gradient in entry 9, and d_feat[n, n_feat].
#include "xpr_internal.cuh"

namespace xpr {
namespace {

constexpr unsigned kFullF = 0xffffffffu;
constexpr int kFeatBatch = 128;

// pixels per thread: 4 up to 2 channels, else 2 (each pixel keeps NF values; at one pixel per
// thread the 16-channel adjoint's per-entry warp reduction served only 32 pixels and ran 1.33 ms on
// the headline against 0.97 ms at two), and no more than a whole-warp block allows
template <int TW, int TH, int NF>
__host__ __device__ constexpr int feat_px() {
    constexpr int want = NF <= 2 ? 4 : 2;
    constexpr int cap = (TW * TH) / 32 >= 4 ? 4 : (TW * TH) / 32;
    return want < cap ? want : cap;
}

struct FeatConsts {
    int W, H, Wt, T;
    uint32_t n;
    int batch;
    float at, amax, teps, bg0, bg1, bg2;
    int nfeat, depth;  // user channels; 1 if the depth channel follows them
};

template <int NF>
__device__ __forceinline__ void feat_stage(const float *__restrict__ rec, const float *__restrict__ feat,
                                           const uint32_t *__restrict__ vals, int e, const FeatConsts &k,
                                           float4 *s_g, float4 *s_c, float *s_b, float (*s_f)[NF], uint32_t *s_id,
                                           int slot) {
    const uint32_t id = __ldg(vals + e);
    const bool ok = id < k.n;
    const Shade s = ok ? load_shade(rec, id) : Shade{0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    s_g[slot] = make_float4(s.mx, s.my, s.A, s.B);
    s_c[slot] = make_float4(s.C, s.o, s.r, s.g);
    s_b[slot] = s.b;
#pragma unroll
    for (int c = 0; c < NF; ++c) {
        float v = 0.f;
        if (ok && c < k.nfeat) v = __ldg(feat + (size_t)id * k.nfeat + c);
        else if (ok && k.depth && c == k.nfeat) v = __ldg(rec + (size_t)id * XPR_REC_FLOATS + 9);
        s_f[slot][c] = v;
    }
    if (s_id) s_id[slot] = id;
}

template <int NF>
struct FPixFwd {
    float fy, T, r, g, b, f[NF];
    int last;
    bool done;
};

template <int TW, int TH, int NF>
__global__ void __launch_bounds__(TW *TH / feat_px<TW, TH, NF>()) render_feat_fwd_kernel(
    const float *__restrict__ rec, const float *__restrict__ feat, const uint32_t *__restrict__ vals,
    const int2 *__restrict__ ranges, FeatConsts k, float *__restrict__ image, float *__restrict__ features,
    float *__restrict__ tfin, int *__restrict__ ncon) {
    grid_dep_wait();
    constexpr int PX = feat_px<TW, TH, NF>();
    constexpr int NT = TW * TH / PX, RS = TH / PX;
    static_assert(NT % 32 == 0, "a tile's block must be whole warps");
    __shared__ float4 s_g[kFeatBatch], s_c[kFeatBatch];
    __shared__ float s_b[kFeatBatch];
    __shared__ float s_f[kFeatBatch][NF];
    const int tile = blockIdx.x;
    const int tx = tile % k.Wt, ty = tile / k.Wt;
    const int t = threadIdx.x;
    const int px = tx * TW + t % TW, py = ty * TH + t / TW;
    const int2 rg = ranges[tile];
    const float fx = (float)px;
    FPixFwd<NF> P[PX];
    bool in[PX];
    bool all_done = true;
#pragma unroll
    for (int q = 0; q < PX; ++q) {
        in[q] = px < k.W && py + q * RS < k.H;
        P[q].fy = (float)(py + q * RS);
        P[q].T = 1.f;
        P[q].r = P[q].g = P[q].b = 0.f;
#pragma unroll
        for (int c = 0; c < NF; ++c) P[q].f[c] = 0.f;
        P[q].last = 0;
        P[q].done = !in[q];
        all_done &= P[q].done;
    }
    for (int base = rg.x; base < rg.y; base += k.batch) {
        if (__syncthreads_and(all_done)) break;
        const int cnt = min(k.batch, rg.y - base);
        for (int e = t; e < cnt; e += NT) feat_stage<NF>(rec, feat, vals, base + e, k, s_g, s_c, s_b, s_f, nullptr, e);
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
                for (int q = 0; q < PX; ++q) {
                    // the colour forward's gates and blend (render.cu), so the image is identical
                    FPixFwd<NF> &p = P[q];
                    const float dy = __fsub_rn(p.fy, g.y);
                    const float pw = eval_power2(ct, c.x, dy);
                    const float og = __fmul_rn(c.y, ex2_approx(pw));
                    const float al = fminf(k.amax, og);
                    const bool live = !p.done && pw <= 0.f && al >= k.at;
                    const float tt = __fmul_rn(p.T, __fsub_rn(1.f, al));
                    const bool stop = live && tt < k.teps;
                    if (live && !stop) {
                        const float w = al * p.T;
                        p.r = fmaf(c.z, w, p.r);
                        p.g = fmaf(c.w, w, p.g);
                        p.b = fmaf(cb, w, p.b);
#pragma unroll
                        for (int ch = 0; ch < NF; ++ch) p.f[ch] = fmaf(s_f[j][ch], w, p.f[ch]);
                        p.T = tt;
                        p.last = pos + 1;
                    }
                    p.done = p.done || stop;
                    all_done &= p.done;
                }
                if (all_done) break;
            }
        }
    }
    const int64_t HW = (int64_t)k.W * k.H;
    const int nf = k.nfeat + k.depth;
#pragma unroll
    for (int q = 0; q < PX; ++q) {
        if (!in[q]) continue;
        const int64_t pix = (int64_t)(py + q * RS) * k.W + px;
        image[pix] = fmaf(P[q].T, k.bg0, P[q].r);
        image[HW + pix] = fmaf(P[q].T, k.bg1, P[q].g);
        image[2 * HW + pix] = fmaf(P[q].T, k.bg2, P[q].b);
#pragma unroll
        for (int ch = 0; ch < NF; ++ch)
            if (ch < nf) features[ch * HW + pix] = P[q].f[ch];
        tfin[pix] = P[q].T;
        ncon[pix] = P[q].last;
    }
}

// 32 per-lane values summed over the warp with 31 shuffles; returns value `lane`
__device__ __forceinline__ float reduce_scatter32f(const float *v, int lane) {
    float b[16];
#pragma unroll
    for (int q = 0; q < 16; ++q) {
        const bool u = lane & 16;
        b[q] = (u ? v[q + 16] : v[q]) + __shfl_xor_sync(kFullF, u ? v[q] : v[q + 16], 16);
    }
    float c[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        const bool u = lane & 8;
        c[q] = (u ? b[q + 8] : b[q]) + __shfl_xor_sync(kFullF, u ? b[q] : b[q + 8], 8);
    }
    float d[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const bool u = lane & 4;
        d[q] = (u ? c[q + 4] : c[q]) + __shfl_xor_sync(kFullF, u ? c[q] : c[q + 4], 4);
    }
    float e[2];
#pragma unroll
    for (int q = 0; q < 2; ++q) {
        const bool u = lane & 2;
        e[q] = (u ? d[q + 2] : d[q]) + __shfl_xor_sync(kFullF, u ? d[q] : d[q + 2], 2);
    }
    const bool u = lane & 1;
    return (u ? e[1] : e[0]) + __shfl_xor_sync(kFullF, u ? e[0] : e[1], 1);
}

template <int NF>
struct FPixBwd {
    float fy, T, g0, g1, g2, B, gf[NF];  // B = sum over channels of g . (value behind the entry)
    int last;
};

// partials into v[32]: v[0..8] as the colour-only adjoint (base-2 form), v[9 + c] dL/df_c
template <int NF>
__device__ __forceinline__ bool feat_adjoint(FPixBwd<NF> &P, float dx, const ColTerms &ct, const float4 &g,
                                             const float4 &c, float cb, const float *f, int pos, const FeatConsts &k,
                                             float *v) {
    if (pos >= P.last) return false;
    const float dy = __fsub_rn(P.fy, g.y);
    const float p = eval_power2(ct, c.x, dy);
    if (p > 0.f) return false;
    const float G = ex2_approx(p);
    const float og = __fmul_rn(c.y, G);
    const float al = fminf(k.amax, og);
    if (al < k.at) return false;
    const float inv = rcp_approx(1.f - al);
    const float Ti = P.T * inv;
    const float w = al * Ti;
    v[6] = fmaf(P.g0, w, v[6]);
    v[7] = fmaf(P.g1, w, v[7]);
    v[8] = fmaf(P.g2, w, v[8]);
    float gc = fmaf(P.g0, c.z, fmaf(P.g1, c.w, P.g2 * cb));
#pragma unroll
    for (int ch = 0; ch < NF; ++ch) {
        gc = fmaf(P.gf[ch], f[ch], gc);
        v[9 + ch] = fmaf(P.gf[ch], w, v[9 + ch]);
    }
    const float dal = fmaf(gc, Ti, -P.B * inv);
    P.B = fmaf(gc, w, P.B);
    P.T = Ti;
    if (og < k.amax) {
        const float dp = dal * al;
        v[5] = fmaf(dal, G, v[5]);
        v[0] = fmaf(dp, fmaf(2.f * g.z, dx, g.w * dy), v[0]);
        v[1] = fmaf(dp, fmaf(g.w, dx, 2.f * c.x * dy), v[1]);
        v[2] = fmaf(dp * dx, dx, v[2]);
        v[3] = fmaf(dp * dx, dy, v[3]);
        v[4] = fmaf(dp * dy, dy, v[4]);
    }
    return true;
}

template <int TW, int TH, int NF>
__global__ void __launch_bounds__(TW *TH / feat_px<TW, TH, NF>()) render_feat_bwd_kernel(
    const float *__restrict__ rec, const float *__restrict__ feat, const uint32_t *__restrict__ vals,
    const int2 *__restrict__ ranges, FeatConsts k, const float *__restrict__ tfin, const int *__restrict__ ncon,
    const float *__restrict__ dimg, const float *__restrict__ dfeat_img, float *__restrict__ d_rec,
    float *__restrict__ d_feat) {
    grid_dep_wait();
    constexpr int PX = feat_px<TW, TH, NF>();
    constexpr int NT = TW * TH / PX, NW = NT / 32, RS = TH / PX;
    constexpr int NV = 9 + NF;
    static_assert(NV <= 32, "at most 23 feature channels per launch");
    __shared__ float4 s_g[kFeatBatch], s_c[kFeatBatch];
    __shared__ float s_b[kFeatBatch];
    __shared__ float s_f[kFeatBatch][NF];
    __shared__ uint32_t s_id[kFeatBatch];
    __shared__ float s_acc[NV][kFeatBatch + 1];  // padded rows: the adding lanes hit different banks
    __shared__ int s_wmax[NW];
    const int tile = blockIdx.x;
    const int tx = tile % k.Wt, ty = tile / k.Wt;
    const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
    const int px = tx * TW + t % TW, py = ty * TH + t / TW;
    const int2 rg = ranges[tile];
    const float fx = (float)px;
    const int64_t HW = (int64_t)k.W * k.H;
    const int nf = k.nfeat + k.depth;
    FPixBwd<NF> P[PX];
    int mylast = 0;
#pragma unroll
    for (int q = 0; q < PX; ++q) {
        const int y = py + q * RS;
        const bool in = px < k.W && y < k.H;
        const int64_t pix = (int64_t)y * k.W + px;
        P[q].fy = (float)y;
        P[q].T = 1.f;
        P[q].last = 0;
        P[q].g0 = P[q].g1 = P[q].g2 = 0.f;
#pragma unroll
        for (int ch = 0; ch < NF; ++ch) P[q].gf[ch] = (in && ch < nf) ? dfeat_img[ch * HW + pix] : 0.f;
        if (in) {
            P[q].T = tfin[pix];
            P[q].last = ncon[pix];
            P[q].g0 = dimg[pix];
            P[q].g1 = dimg[HW + pix];
            P[q].g2 = dimg[2 * HW + pix];
        }
        P[q].B = P[q].T * fmaf(P[q].g0, k.bg0, fmaf(P[q].g1, k.bg1, P[q].g2 * k.bg2));
        mylast = max(mylast, P[q].last);
    }
    const int wlast = __reduce_max_sync(kFullF, mylast);
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
            feat_stage<NF>(rec, feat, vals, start + e, k, s_g, s_c, s_b, s_f, s_id, e);
#pragma unroll
            for (int c = 0; c < NV; ++c) s_acc[c][e] = 0.f;
        }
        __syncthreads();
        for (int j = cnt - 1; j >= 0; --j) {
            const int pos = start + j - rg.x;
            if (pos >= wlast) continue;  // warp-uniform
            float vv[32];
#pragma unroll
            for (int c = 0; c < 32; ++c) vv[c] = 0.f;
            const float4 g = s_g[j];
            const float4 c = s_c[j];
            const float cb = s_b[j];
            float f[NF];
#pragma unroll
            for (int ch = 0; ch < NF; ++ch) f[ch] = s_f[j][ch];
            const float dx = __fsub_rn(fx, g.x);
            const ColTerms ct = column_terms(g.z, g.w, dx);
            bool hit = false;
#pragma unroll
            for (int q = 0; q < PX; ++q) hit |= feat_adjoint<NF>(P[q], dx, ct, g, c, cb, f, pos, k, vv);
            if (__any_sync(kFullF, hit)) {
                const float r = reduce_scatter32f(vv, lane);
                if (lane < NV) atomicAdd(&s_acc[lane][j], r);
            }
        }
        __syncthreads();
        for (int e = t; e < cnt; e += NT) {
            float a[NV];
            bool any = false;
#pragma unroll
            for (int c = 0; c < NV; ++c) {
                a[c] = s_acc[c][e];
                any |= (a[c] != 0.f);
            }
            if (!any || s_id[e] >= k.n) continue;
            const uint32_t id = s_id[e];
            float4 *d = reinterpret_cast<float4 *>(d_rec + (size_t)id * XPR_REC_FLOATS);
            atomicAdd(d, make_float4(-kLn2 * a[0], -kLn2 * a[1], -0.5f * a[2], -a[3]));
            atomicAdd(d + 1, make_float4(-0.5f * a[4], a[5], a[6], a[7]));
            atomicAdd(reinterpret_cast<float *>(d + 2), a[8]);
            if (k.depth) atomicAdd(reinterpret_cast<float *>(d + 2) + 1, a[9 + k.nfeat]);
#pragma unroll
            for (int ch = 0; ch < NF; ++ch)
                if (ch < k.nfeat && a[9 + ch] != 0.f) atomicAdd(d_feat + (size_t)id * k.nfeat + ch, a[9 + ch]);
        }
    }
}

FeatConsts make_feat_consts(const XprCamera &cam, const XprConfig &cfg, int64_t n, int nfeat, int depth) {
    FeatConsts k;
    k.n = (uint32_t)n;
    k.W = cam.width;
    k.H = cam.height;
    k.Wt = tiles_x(cam, cfg);
    k.T = tiles_x(cam, cfg) * tiles_y(cam, cfg);
    k.batch = cfg.batch_depth > 0 ? min(cfg.batch_depth, kFeatBatch) : kFeatBatch;
    k.at = cfg.alpha_thresh;
    k.amax = cfg.alpha_max;
    k.teps = cfg.t_eps;
    k.bg0 = cfg.bg[0];
    k.bg1 = cfg.bg[1];
    k.bg2 = cfg.bg[2];
    k.nfeat = nfeat;
    k.depth = depth ? 1 : 0;
    return k;
}

#define XPR_FEAT_NF_DISPATCH(NFV, nf, ...)                          \
    if ((nf) <= 1) { constexpr int NFV = 1; __VA_ARGS__; }           \
    else if ((nf) <= 2) { constexpr int NFV = 2; __VA_ARGS__; }      \
    else if ((nf) <= 4) { constexpr int NFV = 4; __VA_ARGS__; }      \
    else if ((nf) <= 8) { constexpr int NFV = 8; __VA_ARGS__; }      \
    else if ((nf) <= 12) { constexpr int NFV = 12; __VA_ARGS__; }    \
    else { constexpr int NFV = 16; __VA_ARGS__; }

#define XPR_FEAT_TILE_DISPATCH(TWV, THV, ...)                                                     \
    if (cfg.tile_w == 16 && cfg.tile_h == 16) { constexpr int TWV = 16, THV = 16; __VA_ARGS__; }  \
    else if (cfg.tile_w == 8 && cfg.tile_h == 8) { constexpr int TWV = 8, THV = 8; __VA_ARGS__; } \
    else if (cfg.tile_w == 16 && cfg.tile_h == 8) { constexpr int TWV = 16, THV = 8; __VA_ARGS__; } \
    else { constexpr int TWV = 8, THV = 16; __VA_ARGS__; }

}  // namespace

int launch_render_feat_fwd(const float *rec, int64_t n, const float *feat, int nfeat, int depth, const uint32_t *vals,
                           const int32_t *ranges, const XprCamera &cam, const XprConfig &cfg, float *image,
                           float *features, float *t_final, int32_t *n_contrib, cudaStream_t st) {
    const FeatConsts k = make_feat_consts(cam, cfg, n, nfeat, depth);
    if (k.T == 0) return XPR_OK;
    const int2 *rg = reinterpret_cast<const int2 *>(ranges);
    const int nf = nfeat + (depth ? 1 : 0);
    XPR_FEAT_TILE_DISPATCH(TW, TH, XPR_FEAT_NF_DISPATCH(NF, nf, {
        XPR_CUDA_TRY(launch_dependent(render_feat_fwd_kernel<TW, TH, NF>, dim3(k.T),
                                      dim3(TW * TH / feat_px<TW, TH, NF>()), 0, st, rec, feat, vals, rg, k, image,
                                      features, t_final, n_contrib));
    }));
    XPR_LAUNCH_CHECK("render_feat_fwd_kernel");
    return XPR_OK;
}

int launch_render_feat_bwd(const float *rec, int64_t n, const float *feat, int nfeat, int depth, const uint32_t *vals,
                           const int32_t *ranges, const XprCamera &cam, const XprConfig &cfg, const float *t_final,
                           const int32_t *n_contrib, const float *d_image, const float *d_features, float *d_rec,
                           float *d_feat, cudaStream_t st) {
    XPR_CUDA_TRY(cudaMemsetAsync(d_rec, 0, (size_t)n * XPR_REC_FLOATS * sizeof(float), st));
    if (nfeat > 0) XPR_CUDA_TRY(cudaMemsetAsync(d_feat, 0, (size_t)n * nfeat * sizeof(float), st));
    const FeatConsts k = make_feat_consts(cam, cfg, n, nfeat, depth);
    if (k.T == 0) return XPR_OK;
    const int2 *rg = reinterpret_cast<const int2 *>(ranges);
    const int nf = nfeat + (depth ? 1 : 0);
    XPR_FEAT_TILE_DISPATCH(TW, TH, XPR_FEAT_NF_DISPATCH(NF, nf, {
        XPR_CUDA_TRY(launch_dependent(render_feat_bwd_kernel<TW, TH, NF>, dim3(k.T),
                                      dim3(TW * TH / feat_px<TW, TH, NF>()), 0, st, rec, feat, vals, rg, k, t_final,
                                      n_contrib, d_image, d_features, d_rec, d_feat));
    }));
    XPR_LAUNCH_CHECK("render_feat_bwd_kernel");
    return XPR_OK;
}

}  // namespace xpr
