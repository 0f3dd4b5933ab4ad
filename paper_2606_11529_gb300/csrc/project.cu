// Preprocess stage: 3DGS projection (K1) and its adjoint (K6), for one or several views.
//
// Forward (Listing 1 project; Sec. 2 Preprocess; Appendix 3DGS implementation):
//   camera point  m_c = W mu + t
//   Sigma         = R S S^T R^T          (R from the normalised quaternion, S = diag(s))
//   EWA           Sigma_2D = J W Sigma W^T J^T + dilation I,  J = d(pixel)/d(m_c) with x/z, y/z
//                 clamped to clip_factor x half field of view
//   conic         = Sigma_2D^{-1}
//   extents       ex = sqrt(2 ln(o/a_t) Sigma_2D,xx), ey likewise  (opacity-aware)
//   bounding box  [floor((mx-ex)/w), floor((mx+ex)/w)+1) x (same in y), clamped to the tile grid
//   visible       det > 0 & o >= a_t & r > 0 & tc > 0 & z > z_near
//   colour        max(0, sum_k sh_k Y_k(d) + 0.5),  d = (mu - camera centre) / |.|
// One thread per primitive reads its parameters once and projects them for every view of the
// launch (records of view v at v * n + i); optionally it also counts the tiles of each box that
// pass the tile cull (cull.cuh), so the binning needs no counting pass.
//
// Adjoint (K6): recomputes the forward quantities per view and sums the per-view gradients in
// registers before one write per parameter.  Kernels are instantiated per SH degree so the
// basis loops are static.
#include "cull.cuh"

namespace xpr {
namespace {

// Real spherical harmonics up to degree 3 (Condon-Shortley phase), as polynomials of the
// unit direction.  Constants: C0 = 1/(2 sqrt(pi)), C1 = sqrt(3/(4 pi)),
// C2 = {sqrt(15/pi)/2, -sqrt(15/pi)/2, sqrt(5/pi)/4, -sqrt(15/pi)/2, sqrt(15/pi)/4},
// C3 = {-sqrt(35/(2 pi))/4, sqrt(105/pi)/2, -sqrt(21/(2 pi))/4, sqrt(7/pi)/4,
//       -sqrt(21/(2 pi))/4, sqrt(105/pi)/4, -sqrt(35/(2 pi))/4}.
constexpr float kC0 = 0.28209479177387814f;
constexpr float kC1 = 0.4886025119029199f;
constexpr float kC2a = 1.0925484305920792f;
constexpr float kC2b = 0.31539156525252005f;
constexpr float kC2c = 0.5462742152960396f;
constexpr float kC3a = 0.5900435899266435f;
constexpr float kC3b = 2.890611442640554f;
constexpr float kC3c = 0.4570457994644658f;
constexpr float kC3d = 0.3731763325901154f;
constexpr float kC3e = 1.445305721320277f;

template <int DEG>
__device__ __forceinline__ void sh_basis(float x, float y, float z, float *Y) {
    Y[0] = kC0;
    if constexpr (DEG >= 1) {
        Y[1] = -kC1 * y;
        Y[2] = kC1 * z;
        Y[3] = -kC1 * x;
    }
    if constexpr (DEG >= 2) {
        const float xx = x * x, yy = y * y, zz = z * z;
        Y[4] = kC2a * x * y;
        Y[5] = -kC2a * y * z;
        Y[6] = kC2b * (2.f * zz - xx - yy);
        Y[7] = -kC2a * x * z;
        Y[8] = kC2c * (xx - yy);
        if constexpr (DEG >= 3) {
            Y[9] = -kC3a * y * (3.f * xx - yy);
            Y[10] = kC3b * x * y * z;
            Y[11] = -kC3c * y * (4.f * zz - xx - yy);
            Y[12] = kC3d * z * (2.f * zz - 3.f * xx - 3.f * yy);
            Y[13] = -kC3c * x * (4.f * zz - xx - yy);
            Y[14] = kC3e * z * (xx - yy);
            Y[15] = -kC3a * x * (xx - 3.f * yy);
        }
    }
}

// Partial derivatives of the polynomials above w.r.t. (x, y, z); G[k] = (dYk/dx, dYk/dy, dYk/dz).
template <int DEG>
__device__ __forceinline__ void sh_basis_grad(float x, float y, float z, float3 *G) {
    G[0] = make_float3(0.f, 0.f, 0.f);
    if constexpr (DEG >= 1) {
        G[1] = make_float3(0.f, -kC1, 0.f);
        G[2] = make_float3(0.f, 0.f, kC1);
        G[3] = make_float3(-kC1, 0.f, 0.f);
    }
    if constexpr (DEG >= 2) {
        const float xx = x * x, yy = y * y, zz = z * z;
        G[4] = make_float3(kC2a * y, kC2a * x, 0.f);
        G[5] = make_float3(0.f, -kC2a * z, -kC2a * y);
        G[6] = make_float3(-2.f * kC2b * x, -2.f * kC2b * y, 4.f * kC2b * z);
        G[7] = make_float3(-kC2a * z, 0.f, -kC2a * x);
        G[8] = make_float3(2.f * kC2c * x, -2.f * kC2c * y, 0.f);
        if constexpr (DEG >= 3) {
            G[9] = make_float3(-kC3a * 6.f * x * y, -kC3a * (3.f * xx - 3.f * yy), 0.f);
            G[10] = make_float3(kC3b * y * z, kC3b * x * z, kC3b * x * y);
            G[11] = make_float3(kC3c * 2.f * x * y, -kC3c * (4.f * zz - xx - 3.f * yy), -kC3c * 8.f * y * z);
            G[12] = make_float3(-kC3d * 6.f * x * z, -kC3d * 6.f * y * z, kC3d * (6.f * zz - 3.f * xx - 3.f * yy));
            G[13] = make_float3(-kC3c * (4.f * zz - 3.f * xx - yy), kC3c * 2.f * x * y, -kC3c * 8.f * x * z);
            G[14] = make_float3(kC3e * 2.f * x * z, -kC3e * 2.f * y * z, kC3e * (xx - yy));
            G[15] = make_float3(-kC3a * (3.f * xx - 3.f * yy), kC3a * 6.f * x * y, 0.f);
        }
    }
}

struct Cam {
    float W[9], t[3], cpos[3];
    float fx, fy, cx, cy, limx, limy, z_near;
    int width, height;
};

__device__ __forceinline__ Cam make_cam(const XprCamera &c, const XprConfig &g) {
    Cam k;
    for (int i = 0; i < 3; ++i) {
        for (int j = 0; j < 3; ++j) k.W[3 * i + j] = c.viewmat[4 * i + j];
        k.t[i] = c.viewmat[4 * i + 3];
    }
    for (int i = 0; i < 3; ++i) k.cpos[i] = -(k.W[i] * k.t[0] + k.W[3 + i] * k.t[1] + k.W[6 + i] * k.t[2]);
    k.fx = c.fx;
    k.fy = c.fy;
    k.cx = c.cx;
    k.cy = c.cy;
    k.limx = g.clip_factor * (0.5f * (float)c.width / c.fx);
    k.limy = g.clip_factor * (0.5f * (float)c.height / c.fy);
    k.z_near = c.z_near;
    k.width = c.width;
    k.height = c.height;
    return k;
}

__device__ __forceinline__ void quat_to_rot(float w, float x, float y, float z, float *R) {
    R[0] = 1.f - 2.f * (y * y + z * z);
    R[1] = 2.f * (x * y - w * z);
    R[2] = 2.f * (x * z + w * y);
    R[3] = 2.f * (x * y + w * z);
    R[4] = 1.f - 2.f * (x * x + z * z);
    R[5] = 2.f * (y * z - w * x);
    R[6] = 2.f * (x * z - w * y);
    R[7] = 2.f * (y * z + w * x);
    R[8] = 1.f - 2.f * (x * x + y * y);
}

struct Params {
    float m[3], s[3], q[4], o;
};

__device__ __forceinline__ Params load_params(const float *__restrict__ mu, const float *__restrict__ scale,
                                              const float *__restrict__ quat, const float *__restrict__ opac,
                                              int64_t i) {
    Params P;
    for (int j = 0; j < 3; ++j) {
        P.m[j] = mu[3 * i + j];
        P.s[j] = scale[3 * i + j];
    }
    const float4 q4 = __ldg(reinterpret_cast<const float4 *>(quat) + i);
    P.q[0] = q4.x;
    P.q[1] = q4.y;
    P.q[2] = q4.z;
    P.q[3] = q4.w;
    P.o = opac[i];
    return P;
}

// Forward quantities shared by K1 and K6 (recomputed in K6 instead of stored).
struct Geo {
    float mc[3];
    float qn[4], qinv;
    float R[9];
    float Sig[6];  // xx, xy, xz, yy, yz, zz
    float ux, uy;
    bool clx, cly;
    float T[6];    // J W, 2x3
    float a, b, c; // Sigma_2D (dilated)
    float det;
    float mx, my;
};

__device__ __forceinline__ void geometry(const Params &P, const Cam &k, float dil, Geo &G) {
    for (int i = 0; i < 3; ++i)
        G.mc[i] = k.W[3 * i] * P.m[0] + k.W[3 * i + 1] * P.m[1] + k.W[3 * i + 2] * P.m[2] + k.t[i];
    const float qq = P.q[0] * P.q[0] + P.q[1] * P.q[1] + P.q[2] * P.q[2] + P.q[3] * P.q[3];
    G.qinv = rsqrtf(qq);
    for (int i = 0; i < 4; ++i) G.qn[i] = P.q[i] * G.qinv;
    quat_to_rot(G.qn[0], G.qn[1], G.qn[2], G.qn[3], G.R);
    float M[9];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) M[3 * i + j] = G.R[3 * i + j] * P.s[j];
    G.Sig[0] = M[0] * M[0] + M[1] * M[1] + M[2] * M[2];
    G.Sig[1] = M[0] * M[3] + M[1] * M[4] + M[2] * M[5];
    G.Sig[2] = M[0] * M[6] + M[1] * M[7] + M[2] * M[8];
    G.Sig[3] = M[3] * M[3] + M[4] * M[4] + M[5] * M[5];
    G.Sig[4] = M[3] * M[6] + M[4] * M[7] + M[5] * M[8];
    G.Sig[5] = M[6] * M[6] + M[7] * M[7] + M[8] * M[8];
    const float x = G.mc[0], y = G.mc[1], z = G.mc[2];
    const float iz = 1.f / z;
    const float rx = x * iz, ry = y * iz;
    G.ux = fminf(fmaxf(rx, -k.limx), k.limx);
    G.uy = fminf(fmaxf(ry, -k.limy), k.limy);
    G.clx = (rx < -k.limx) || (rx > k.limx);
    G.cly = (ry < -k.limy) || (ry > k.limy);
    const float J00 = k.fx * iz, J02 = -k.fx * G.ux * iz, J11 = k.fy * iz, J12 = -k.fy * G.uy * iz;
    for (int j = 0; j < 3; ++j) {
        G.T[j] = J00 * k.W[j] + J02 * k.W[6 + j];
        G.T[3 + j] = J11 * k.W[3 + j] + J12 * k.W[6 + j];
    }
    // Sigma_2D' = T Sigma T^T
    const float *T0 = G.T, *T1 = G.T + 3;
    const float *S = G.Sig;
    const float u0[3] = {S[0] * T0[0] + S[1] * T0[1] + S[2] * T0[2], S[1] * T0[0] + S[3] * T0[1] + S[4] * T0[2],
                         S[2] * T0[0] + S[4] * T0[1] + S[5] * T0[2]};
    const float u1[3] = {S[0] * T1[0] + S[1] * T1[1] + S[2] * T1[2], S[1] * T1[0] + S[3] * T1[1] + S[4] * T1[2],
                         S[2] * T1[0] + S[4] * T1[1] + S[5] * T1[2]};
    G.a = T0[0] * u0[0] + T0[1] * u0[1] + T0[2] * u0[2] + dil;
    G.b = T0[0] * u1[0] + T0[1] * u1[1] + T0[2] * u1[2];
    G.c = T1[0] * u1[0] + T1[1] * u1[1] + T1[2] * u1[2] + dil;
    G.det = G.a * G.c - G.b * G.b;
    G.mx = k.fx * rx + k.cx;
    G.my = k.fy * ry + k.cy;
}

struct Footprint {
    bool vis;
    float lt;
    int4 bb;
    int tc;
};

// Visibility flag, ln(o/a_t) and tile bounding box (identical in K1 and K6).
__device__ __forceinline__ Footprint footprint(const Geo &G, float o, const Cam &k, const XprConfig &cfg) {
    Footprint f;
    f.vis = (G.mc[2] > k.z_near) && (G.det > 0.f) && (o >= cfg.alpha_thresh);
    f.lt = 0.f;
    f.bb = make_int4(0, 0, 0, 0);
    f.tc = 0;
    if (f.vis) {
        f.lt = logf(o / cfg.alpha_thresh);
        const float ex = sqrtf(2.f * f.lt * G.a);
        const float ey = sqrtf(2.f * f.lt * G.c);
        const float Wt = (float)((k.width + cfg.tile_w - 1) / cfg.tile_w);
        const float Ht = (float)((k.height + cfg.tile_h - 1) / cfg.tile_h);
        const float tw = (float)cfg.tile_w, th = (float)cfg.tile_h;
        f.bb.x = (int)fminf(fmaxf(floorf((G.mx - ex) / tw), 0.f), Wt);
        f.bb.y = (int)fminf(fmaxf(floorf((G.my - ey) / th), 0.f), Ht);
        f.bb.z = (int)fminf(fmaxf(floorf((G.mx + ex) / tw) + 1.f, 0.f), Wt);
        f.bb.w = (int)fminf(fmaxf(floorf((G.my + ey) / th) + 1.f, 0.f), Ht);
        f.tc = (f.bb.z - f.bb.x) * (f.bb.w - f.bb.y);
        f.vis = (fmaxf(ex, ey) > 0.f) && (f.tc > 0);
    }
    return f;
}

struct CamSet {
    XprCamera cam[kMaxViews];
    int n_views;
};

// K1 for one view: writes rec / bbox / tile count of record `out` and returns the cull data.
// View-dependent colour (before the clamp at 0): 0.5 + sum_k sh_k Y_k(d), d = unit vector from the
// camera centre to the mean.
template <int DEG>
__device__ __forceinline__ void sh_colour(const Params &P, const float *shi, const Cam &k, float *col) {
    constexpr int K = (DEG + 1) * (DEG + 1);
    const float vx = P.m[0] - k.cpos[0], vy = P.m[1] - k.cpos[1], vz = P.m[2] - k.cpos[2];
    const float vinv = rsqrtf(vx * vx + vy * vy + vz * vz);
    float Y[K];
    sh_basis<DEG>(vx * vinv, vy * vinv, vz * vinv, Y);
    col[0] = col[1] = col[2] = 0.5f;
#pragma unroll
    for (int kk = 0; kk < K; ++kk) {
        col[0] += shi[3 * kk] * Y[kk];
        col[1] += shi[3 * kk + 1] * Y[kk];
        col[2] += shi[3 * kk + 2] * Y[kk];
    }
}

template <int DEG>
__device__ __forceinline__ void project_view(const Params &P, const float *shi, int64_t out,
                                             const XprCamera &cam, const XprConfig &cfg, float *__restrict__ rec,
                                             int4 *__restrict__ bbox, int *__restrict__ tcount, CullData &cd,
                                             int4 &bb, int &area) {
    const Cam k = make_cam(cam, cfg);
    float col[3] = {0.f, 0.f, 0.f};
    if (shi) sh_colour<DEG>(P, shi, k, col);
    Geo G;
    geometry(P, k, cfg.cov_dilation, G);
    const float z = G.mc[2];
    float4 *o4 = reinterpret_cast<float4 *>(rec + (size_t)out * XPR_REC_FLOATS);
    const Footprint f = footprint(G, P.o, k, cfg);
    if (f.vis) {
        const float idet = 1.f / G.det;
        // the stored record values are the ones the cull reads back, so the count taken here from
        // registers and the emit kernel's decisions from memory are bit-identical
        const float c0 = G.c * idet, c1 = -G.b * idet, c2 = G.a * idet;
        cd = make_cull(G.mx, G.my, c0, c1, c2, f.lt);
        o4[0] = make_float4(G.mx, G.my, c0, c1);
        o4[1] = make_float4(c2, P.o, fmaxf(col[0], 0.f), fmaxf(col[1], 0.f));
        o4[2] = make_float4(fmaxf(col[2], 0.f), z, f.lt, 1.f);
        bbox[out] = f.bb;
        tcount[out] = f.tc;
        bb = f.bb;
        area = f.tc;
    } else {
        o4[0] = make_float4(0.f, 0.f, 0.f, 0.f);
        o4[1] = make_float4(0.f, 0.f, 0.f, 0.f);
        o4[2] = make_float4(0.f, z, 0.f, 0.f);
        bbox[out] = make_int4(0, 0, 0, 0);
        tcount[out] = 0;
        bb = make_int4(0, 0, 0, 0);
        area = 0;
    }
}

// Shared-memory row stride of one primitive's SH coefficients (odd, so the 32 lanes of a warp
// reading their own rows hit 32 different banks).
template <int DEG>
__host__ __device__ constexpr int sh_ld() {
    return ((DEG + 1) * (DEG + 1) * 3) | 1;
}
constexpr int kProjWarps = 4;

// One thread per primitive and all views; each warp first stages its 32 primitives' SH
// coefficients in shared memory with coalesced loads (a thread's own row is 3K floats long).
// Stages the SH coefficients of a warp's 32 primitives (from base) in shared memory, coalesced.
template <int DEG>
__device__ __forceinline__ void stage_sh(const float *__restrict__ sh, int64_t base, int nv, float *ssh) {
    constexpr int KC = (DEG + 1) * (DEG + 1) * 3;
    constexpr int LD = sh_ld<DEG>();
    const int lane = threadIdx.x & 31;
    const float *gs = sh + base * KC;
    for (int e = lane; e < nv * KC; e += 32) {
        const int pi = e / KC;
        ssh[pi * LD + (e - pi * KC)] = __ldg(gs + e);
    }
    __syncwarp();
}

// COLOR = false (sh NULL): geometry only, colours left 0 for xpr_project_color to fill.
template <int DEG, bool COLOR>
__global__ void __launch_bounds__(kProjWarps * 32) project_fwd_kernel(
    const float *__restrict__ mu, const float *__restrict__ scale, const float *__restrict__ quat,
    const float *__restrict__ opac, const float *__restrict__ sh, int64_t n, CamSet cs, XprConfig cfg,
    float *__restrict__ rec, int4 *__restrict__ bbox, int *__restrict__ tcount, int *__restrict__ isect_count) {
    constexpr int LD = sh_ld<DEG>();
    extern __shared__ float s_fwd[];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t base = ((int64_t)blockIdx.x * kProjWarps + w) * 32;
    if (base >= n) return;
    const int nv = (int)min((int64_t)32, n - base);
    float *ssh = s_fwd + (size_t)w * 32 * LD;
    if (COLOR) stage_sh<DEG>(sh, base, nv, ssh);
    const int64_t i = base + lane;
    const bool valid = i < n;
    Params P = {};
    if (valid) P = load_params(mu, scale, quat, opac, i);
    for (int v = 0; v < cs.n_views; ++v) {
        CullData cd = {};
        int4 bb = make_int4(0, 0, 0, 0);
        int area = 0;
        const int64_t out = (int64_t)v * n + i;
        if (valid)
            project_view<DEG>(P, COLOR ? ssh + lane * LD : nullptr, out, cs.cam[v], cfg, rec, bbox, tcount, cd, bb,
                              area);
        if (isect_count) {  // exact number of kept (primitive, tile) pairs, counted with the binning's cull
            const int cnt = count_kept_tiles(cd, bb, area, make_grid(cs.cam[v], cfg));
            if (valid) isect_count[out] = cnt;
        }
    }
}

// The colours of records already projected without them (rec[6..8] of every visible record).
template <int DEG>
__global__ void __launch_bounds__(kProjWarps * 32) project_color_kernel(const float *__restrict__ mu,
                                                                        const float *__restrict__ sh, int64_t n,
                                                                        CamSet cs, XprConfig cfg,
                                                                        float *__restrict__ rec) {
    constexpr int LD = sh_ld<DEG>();
    extern __shared__ float s_col[];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t base = ((int64_t)blockIdx.x * kProjWarps + w) * 32;
    if (base >= n) return;
    const int nv = (int)min((int64_t)32, n - base);
    float *ssh = s_col + (size_t)w * 32 * LD;
    stage_sh<DEG>(sh, base, nv, ssh);
    const int64_t i = base + lane;
    if (i >= n) return;
    Params P = {};
    P.m[0] = mu[3 * i];
    P.m[1] = mu[3 * i + 1];
    P.m[2] = mu[3 * i + 2];
    for (int v = 0; v < cs.n_views; ++v) {
        float *r = rec + ((size_t)v * n + i) * XPR_REC_FLOATS;
        if (r[11] == 0.f) continue;  // invisible: colour stays 0
        float col[3];
        sh_colour<DEG>(P, ssh + lane * LD, make_cam(cs.cam[v], cfg), col);
        r[6] = fmaxf(col[0], 0.f);
        r[7] = fmaxf(col[1], 0.f);
        r[8] = fmaxf(col[2], 0.f);
    }
}

// Accumulators of the adjoint over views.  The quaternion gradient is kept with respect to the
// normalised quaternion and projected through the normalisation once at the end.
template <int DEG>
struct Acc {
    float mu[3], s[3], qn[4], o;
};

// Sum over k of w_k grad Y_k (the partials of sh_basis_grad, folded into the sum term by term so
// that no per-basis gradient array is kept).
template <int DEG>
__device__ __forceinline__ float3 sh_grad_dot(float x, float y, float z, const float *w) {
    float rx = 0.f, ry = 0.f, rz = 0.f;
    if constexpr (DEG >= 1) {
        ry -= kC1 * w[1];
        rz += kC1 * w[2];
        rx -= kC1 * w[3];
    }
    if constexpr (DEG >= 2) {
        rx += kC2a * (w[4] * y - w[7] * z) + 2.f * x * (kC2c * w[8] - kC2b * w[6]);
        ry += kC2a * (w[4] * x - w[5] * z) - 2.f * y * (kC2b * w[6] + kC2c * w[8]);
        rz += kC2a * (-w[5] * y - w[7] * x) + 4.f * kC2b * z * w[6];
        if constexpr (DEG >= 3) {
            const float xx = x * x, yy = y * y, zz = z * z;
            // G9 = (-6 C3a x y, -C3a (3xx - 3yy), 0)
            rx += -kC3a * 6.f * x * y * w[9];
            ry += -kC3a * (3.f * xx - 3.f * yy) * w[9];
            // G10 = C3b (y z, x z, x y)
            rx += kC3b * y * z * w[10];
            ry += kC3b * x * z * w[10];
            rz += kC3b * x * y * w[10];
            // G11 = (2 C3c x y, -C3c (4zz - xx - 3yy), -8 C3c y z)
            rx += kC3c * 2.f * x * y * w[11];
            ry += -kC3c * (4.f * zz - xx - 3.f * yy) * w[11];
            rz += -kC3c * 8.f * y * z * w[11];
            // G12 = (-6 C3d x z, -6 C3d y z, C3d (6zz - 3xx - 3yy))
            rx += -kC3d * 6.f * x * z * w[12];
            ry += -kC3d * 6.f * y * z * w[12];
            rz += kC3d * (6.f * zz - 3.f * xx - 3.f * yy) * w[12];
            // G13 = (-C3c (4zz - 3xx - yy), 2 C3c x y, -8 C3c x z)
            rx += -kC3c * (4.f * zz - 3.f * xx - yy) * w[13];
            ry += kC3c * 2.f * x * y * w[13];
            rz += -kC3c * 8.f * x * z * w[13];
            // G14 = (2 C3e x z, -2 C3e y z, C3e (xx - yy))
            rx += kC3e * 2.f * x * z * w[14];
            ry += -kC3e * 2.f * y * z * w[14];
            rz += kC3e * (xx - yy) * w[14];
            // G15 = (-C3a (3xx - 3yy), 6 C3a x y, 0)
            rx += -kC3a * (3.f * xx - 3.f * yy) * w[15];
            ry += kC3a * 6.f * x * y * w[15];
        }
    }
    return make_float3(rx, ry, rz);
}

// K6 for one view: chains d_rec = (d mu_2D, d conic, d o, d rgb) back to the parameters:
//   conic = A^{-1}:        dL/dA = -A^{-1} G A^{-1}  (G = dL/dconic, off-diagonal split in two)
//   A = T Sigma T^T + dI:   dL/dSigma = T^T dA T,  dL/dT = 2 dA T Sigma
//   T = J W:                dL/dJ = dL/dT W^T;  J(m_c) with the clamp (clamped coordinate is constant)
//   m_c = W mu + t;  mu_2D = (fx x/z + cx, fy y/z + cy)
//   Sigma = M M^T, M = R diag(s):  dL/dM = 2 dL/dSigma M
//   R(q/|q|):               explicit partials of the rotation matrix
//   colour:                 dL/dsh_k = Y_k g (where unclamped); dL/dd through the basis gradient,
//                           projected on the tangent plane and divided by |mu - camera centre|
template <int DEG>
__device__ __forceinline__ void adjoint_view(const Params &P, const float *shi, float *dsh, const Geo &G,
                                             const Cam &k, float4 d0, float4 d1, float4 d2, Acc<DEG> &A) {
    constexpr int K = (DEG + 1) * (DEG + 1);
    const float dmx = d0.x, dmy = d0.y, g00 = d0.z, g01 = d0.w, g11 = d1.x;
    const float drgb[3] = {d1.z, d1.w, d2.x};
    A.o += d1.y;

    // ---- colour
    const float vx = P.m[0] - k.cpos[0], vy = P.m[1] - k.cpos[1], vz = P.m[2] - k.cpos[2];
    const float vinv = rsqrtf(vx * vx + vy * vy + vz * vz);
    const float ux = vx * vinv, uy = vy * vinv, uz = vz * vinv;
    float wk[K];  // w_k = gc . sh_k, then dL/dd = sum_k w_k grad Y_k
    {
        float Y[K];
        sh_basis<DEG>(ux, uy, uz, Y);
        float raw[3] = {0.5f, 0.5f, 0.5f};
#pragma unroll
        for (int kk = 0; kk < K; ++kk) {
            raw[0] += shi[3 * kk] * Y[kk];
            raw[1] += shi[3 * kk + 1] * Y[kk];
            raw[2] += shi[3 * kk + 2] * Y[kk];
        }
        float gc[3];
        for (int c = 0; c < 3; ++c) gc[c] = raw[c] > 0.f ? drgb[c] : 0.f;
#pragma unroll
        for (int kk = 0; kk < K; ++kk) {
            wk[kk] = gc[0] * shi[3 * kk] + gc[1] * shi[3 * kk + 1] + gc[2] * shi[3 * kk + 2];
            dsh[3 * kk] += Y[kk] * gc[0];
            dsh[3 * kk + 1] += Y[kk] * gc[1];
            dsh[3 * kk + 2] += Y[kk] * gc[2];
        }
    }
    const float3 gdir = sh_grad_dot<DEG>(ux, uy, uz, wk);
    const float dd = gdir.x * ux + gdir.y * uy + gdir.z * uz;
    A.mu[0] += (gdir.x - ux * dd) * vinv;
    A.mu[1] += (gdir.y - uy * dd) * vinv;
    A.mu[2] += (gdir.z - uz * dd) * vinv;

    // ---- mu_2D
    const float x = G.mc[0], y = G.mc[1], z = G.mc[2];
    const float iz = 1.f / z, iz2 = iz * iz;
    float gmc[3];
    gmc[0] = dmx * k.fx * iz;
    gmc[1] = dmy * k.fy * iz;
    gmc[2] = -(dmx * k.fx * x + dmy * k.fy * y) * iz2;

    // ---- conic -> Sigma_2D:  dA = -P G P with P = A^{-1} = [[p, q], [q, r]], G = [[g00, h], [h, g11]]
    const float idet = 1.f / G.det;
    const float p = G.c * idet, qq = -G.b * idet, r = G.a * idet;
    const float h = 0.5f * g01;
    const float ga = -(p * p * g00 + 2.f * p * qq * h + qq * qq * g11);
    const float gb = -(p * qq * g00 + (qq * qq + p * r) * h + qq * r * g11);
    const float gcv = -(qq * qq * g00 + 2.f * qq * r * h + r * r * g11);

    // ---- Sigma_2D' = T Sigma T^T: dSigma = T^T dA T ; dT = 2 dA T Sigma
    const float *T0 = G.T, *T1 = G.T + 3;
    const float *S = G.Sig;
    float gS[6];  // xx, xy, xz, yy, yz, zz of the symmetric gradient
    {
        int idx = 0;
#pragma unroll
        for (int a_ = 0; a_ < 3; ++a_)
#pragma unroll
            for (int b_ = a_; b_ < 3; ++b_)
                gS[idx++] = ga * T0[a_] * T0[b_] + gb * (T0[a_] * T1[b_] + T1[a_] * T0[b_]) + gcv * T1[a_] * T1[b_];
    }
    const float TS0[3] = {T0[0] * S[0] + T0[1] * S[1] + T0[2] * S[2], T0[0] * S[1] + T0[1] * S[3] + T0[2] * S[4],
                          T0[0] * S[2] + T0[1] * S[4] + T0[2] * S[5]};
    const float TS1[3] = {T1[0] * S[0] + T1[1] * S[1] + T1[2] * S[2], T1[0] * S[1] + T1[1] * S[3] + T1[2] * S[4],
                          T1[0] * S[2] + T1[1] * S[4] + T1[2] * S[5]};
    float gT0[3], gT1[3];
    for (int j = 0; j < 3; ++j) {
        gT0[j] = 2.f * (ga * TS0[j] + gb * TS1[j]);
        gT1[j] = 2.f * (gb * TS0[j] + gcv * TS1[j]);
    }
    // T = J W: dJ_rk = sum_b dT_rb W_kb ; only J00, J02, J11, J12 are non-zero
    const float *W = k.W;
    const float gJ00 = gT0[0] * W[0] + gT0[1] * W[1] + gT0[2] * W[2];
    const float gJ02 = gT0[0] * W[6] + gT0[1] * W[7] + gT0[2] * W[8];
    const float gJ11 = gT1[0] * W[3] + gT1[1] * W[4] + gT1[2] * W[5];
    const float gJ12 = gT1[0] * W[6] + gT1[1] * W[7] + gT1[2] * W[8];
    gmc[2] += -k.fx * iz2 * gJ00 - k.fy * iz2 * gJ11;
    if (!G.clx) {
        gmc[0] += -k.fx * iz2 * gJ02;
        gmc[2] += 2.f * k.fx * x * iz2 * iz * gJ02;
    } else {
        gmc[2] += k.fx * G.ux * iz2 * gJ02;
    }
    if (!G.cly) {
        gmc[1] += -k.fy * iz2 * gJ12;
        gmc[2] += 2.f * k.fy * y * iz2 * iz * gJ12;
    } else {
        gmc[2] += k.fy * G.uy * iz2 * gJ12;
    }
    for (int j = 0; j < 3; ++j) A.mu[j] += W[j] * gmc[0] + W[3 + j] * gmc[1] + W[6 + j] * gmc[2];

    // ---- Sigma = M M^T, M = R diag(s): dM = 2 dSigma M
    const float gSf[9] = {gS[0], gS[1], gS[2], gS[1], gS[3], gS[4], gS[2], gS[4], gS[5]};
    float M[9];
    for (int a_ = 0; a_ < 3; ++a_)
        for (int c_ = 0; c_ < 3; ++c_) M[3 * a_ + c_] = G.R[3 * a_ + c_] * P.s[c_];
    float gR[9];
    for (int a_ = 0; a_ < 3; ++a_)
        for (int c_ = 0; c_ < 3; ++c_) {
            const float gM = 2.f * (gSf[3 * a_] * M[c_] + gSf[3 * a_ + 1] * M[3 + c_] + gSf[3 * a_ + 2] * M[6 + c_]);
            A.s[c_] += gM * G.R[3 * a_ + c_];
            gR[3 * a_ + c_] = gM * P.s[c_];
        }
    // ---- R(qn): partials of the unit-quaternion rotation matrix
    const float w = G.qn[0], qx = G.qn[1], qy = G.qn[2], qz = G.qn[3];
    A.qn[0] += 2.f * (-qz * gR[1] + qy * gR[2] + qz * gR[3] - qx * gR[5] - qy * gR[6] + qx * gR[7]);
    A.qn[1] += 2.f * (qy * gR[1] + qz * gR[2] + qy * gR[3] - 2.f * qx * gR[4] - w * gR[5] + qz * gR[6] +
                      w * gR[7] - 2.f * qx * gR[8]);
    A.qn[2] += 2.f * (-2.f * qy * gR[0] + qx * gR[1] + w * gR[2] + qx * gR[3] + qz * gR[5] - w * gR[6] +
                      qz * gR[7] - 2.f * qy * gR[8]);
    A.qn[3] += 2.f * (-2.f * qz * gR[0] - w * gR[1] + qx * gR[2] + w * gR[3] - 2.f * qz * gR[4] + qy * gR[5] +
                      qx * gR[6] + qy * gR[7]);
}

constexpr int kBwdWarps = 4;

// One thread per primitive; each warp stages its 32 primitives' SH coefficients in shared memory
// with coalesced loads and accumulates their gradients there, then writes them out coalesced (a
// thread's own rows are 3K floats apart in global memory).
template <int DEG>
__global__ void __launch_bounds__(kBwdWarps * 32, 4) project_bwd_kernel(
    const float *__restrict__ mu, const float *__restrict__ scale, const float *__restrict__ quat,
    const float *__restrict__ opac, const float *__restrict__ sh, int64_t n, CamSet cs, XprConfig cfg,
    const float *__restrict__ d_rec, float *__restrict__ gmu, float *__restrict__ gscale, float *__restrict__ gquat,
    float *__restrict__ gopac, float *__restrict__ gsh) {
    constexpr int KC = (DEG + 1) * (DEG + 1) * 3;
    constexpr int LD = sh_ld<DEG>();
    extern __shared__ float s_bwd[];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t base = ((int64_t)blockIdx.x * kBwdWarps + w) * 32;
    if (base >= n) return;
    const int nv = (int)min((int64_t)32, n - base);
    float *ssh = s_bwd + (size_t)w * 2 * 32 * LD;
    float *sdsh = ssh + 32 * LD;
    const float *gs = sh + base * KC;
    for (int e = lane; e < nv * KC; e += 32) {
        const int pi = e / KC;
        ssh[pi * LD + (e - pi * KC)] = __ldg(gs + e);
    }
    for (int c = 0; c < KC; ++c) sdsh[lane * LD + c] = 0.f;
    __syncwarp();
    const int64_t i = base + lane;
    if (i < n) {
        const Params P = load_params(mu, scale, quat, opac, i);
        Acc<DEG> A = {};
        float qinv = 0.f, qn[4] = {0.f, 0.f, 0.f, 0.f};
        for (int v = 0; v < cs.n_views; ++v) {
            const Cam k = make_cam(cs.cam[v], cfg);
            Geo G;
            geometry(P, k, cfg.cov_dilation, G);
            if (!footprint(G, P.o, k, cfg).vis) continue;  // invisible in this view: no gradient from it
            const float4 *D4 = reinterpret_cast<const float4 *>(d_rec + ((size_t)v * n + i) * XPR_REC_FLOATS);
            adjoint_view<DEG>(P, ssh + lane * LD, sdsh + lane * LD, G, k, __ldg(D4), __ldg(D4 + 1), __ldg(D4 + 2),
                              A);
            qinv = G.qinv;
            for (int j = 0; j < 4; ++j) qn[j] = G.qn[j];
        }
        // qn = q / |q|:  dL/dq = (dL/dqn - qn (qn . dL/dqn)) / |q|
        const float dot = A.qn[0] * qn[0] + A.qn[1] * qn[1] + A.qn[2] * qn[2] + A.qn[3] * qn[3];
        for (int j = 0; j < 3; ++j) {
            gmu[3 * i + j] = A.mu[j];
            gscale[3 * i + j] = A.s[j];
        }
        reinterpret_cast<float4 *>(gquat)[i] =
            make_float4((A.qn[0] - qn[0] * dot) * qinv, (A.qn[1] - qn[1] * dot) * qinv,
                        (A.qn[2] - qn[2] * dot) * qinv, (A.qn[3] - qn[3] * dot) * qinv);
        gopac[i] = A.o;
    }
    __syncwarp();
    float *go = gsh + base * KC;
    for (int e = lane; e < nv * KC; e += 32) {
        const int pi = e / KC;
        go[e] = sdsh[pi * LD + (e - pi * KC)];
    }
}

CamSet make_camset(const XprCamera *cams, int n_views) {
    CamSet cs;
    memset(&cs, 0, sizeof(cs));
    for (int v = 0; v < n_views; ++v) cs.cam[v] = cams[v];
    cs.n_views = n_views;
    return cs;
}

#define XPR_DEG_DISPATCH(DEGV, ...)                              \
    switch (cfg.sh_degree) {                                     \
        case 0: { constexpr int DEGV = 0; __VA_ARGS__; } break; \
        case 1: { constexpr int DEGV = 1; __VA_ARGS__; } break; \
        case 2: { constexpr int DEGV = 2; __VA_ARGS__; } break; \
        default: { constexpr int DEGV = 3; __VA_ARGS__; } break; \
    }

}  // namespace

int launch_project_fwd_views(const XprPrims &p, int64_t n, const XprCamera *cams, int n_views, const XprConfig &cfg,
                             float *rec, int32_t *bbox, int32_t *tc, int32_t *isect_count, cudaStream_t st) {
    if (n == 0 || n_views == 0) return XPR_OK;
    const int tpb = kProjWarps * 32;
    const unsigned blocks = (unsigned)((n + tpb - 1) / tpb);
    const CamSet cs = make_camset(cams, n_views);
    if (p.sh) {
        XPR_DEG_DISPATCH(DEG, project_fwd_kernel<DEG, true><<<blocks, tpb,
                                                               (size_t)kProjWarps * 32 * sh_ld<DEG>() * sizeof(float),
                                                               st>>>(p.mu, p.scale, p.quat, p.opacity, p.sh, n, cs,
                                                                     cfg, rec, reinterpret_cast<int4 *>(bbox), tc,
                                                                     isect_count));
    } else {
        XPR_DEG_DISPATCH(DEG, project_fwd_kernel<DEG, false><<<blocks, tpb, 0, st>>>(
                                  p.mu, p.scale, p.quat, p.opacity, nullptr, n, cs, cfg, rec,
                                  reinterpret_cast<int4 *>(bbox), tc, isect_count));
    }
    XPR_LAUNCH_CHECK("project_fwd_kernel");
    return XPR_OK;
}

int launch_project_color_views(const float *mu, const float *sh, int64_t n, const XprCamera *cams, int n_views,
                               const XprConfig &cfg, float *rec, cudaStream_t st) {
    if (n == 0 || n_views == 0) return XPR_OK;
    const int tpb = kProjWarps * 32;
    const unsigned blocks = (unsigned)((n + tpb - 1) / tpb);
    const CamSet cs = make_camset(cams, n_views);
    XPR_DEG_DISPATCH(DEG, project_color_kernel<DEG><<<blocks, tpb,
                                                       (size_t)kProjWarps * 32 * sh_ld<DEG>() * sizeof(float), st>>>(
                              mu, sh, n, cs, cfg, rec));
    XPR_LAUNCH_CHECK("project_color_kernel");
    return XPR_OK;
}

int launch_project_bwd_views(const XprPrims &p, int64_t n, const XprCamera *cams, int n_views, const XprConfig &cfg,
                             const float *d_rec, const XprPrimsGrad &g, cudaStream_t st) {
    if (n == 0 || n_views == 0) return XPR_OK;
    const int tpb = kBwdWarps * 32;
    const unsigned blocks = (unsigned)((n + tpb - 1) / tpb);
    const CamSet cs = make_camset(cams, n_views);
    cudaError_t attr = cudaSuccess;
    // the shared-memory size is a constant of each instantiation, so every caller sets the same limit
    XPR_DEG_DISPATCH(DEG, {
        const size_t smem = (size_t)kBwdWarps * 2 * 32 * sh_ld<DEG>() * sizeof(float);
        attr = cudaFuncSetAttribute(project_bwd_kernel<DEG>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (attr == cudaSuccess)
            project_bwd_kernel<DEG><<<blocks, tpb, smem, st>>>(p.mu, p.scale, p.quat, p.opacity, p.sh, n, cs, cfg,
                                                               d_rec, g.mu, g.scale, g.quat, g.opacity, g.sh);
    });
    XPR_CUDA_TRY(attr);
    XPR_LAUNCH_CHECK("project_bwd_kernel");
    return XPR_OK;
}

int launch_project_fwd(const XprPrims &p, int64_t n, const XprCamera &cam, const XprConfig &cfg, float *rec,
                       int32_t *bbox, int32_t *tc, int32_t *isect_count, cudaStream_t st) {
    return launch_project_fwd_views(p, n, &cam, 1, cfg, rec, bbox, tc, isect_count, st);
}

int launch_project_bwd(const XprPrims &p, int64_t n, const XprCamera &cam, const XprConfig &cfg,
                       const float *d_rec, const XprPrimsGrad &g, cudaStream_t st) {
    return launch_project_bwd_views(p, n, &cam, 1, cfg, d_rec, g, st);
}

}  // namespace xpr
