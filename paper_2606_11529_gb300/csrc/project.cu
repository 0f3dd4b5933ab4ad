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
#include "project_common.cuh"

namespace xpr {
namespace {

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
    cam_point(k, P.m, G.mc);
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

// K1 for one view: writes rec / bbox / tile count of record `out` and returns the cull data.
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

// COLOR = false (sh NULL): geometry only, colours left 0 for xpr_project_color to fill.
// copy.mu non-NULL: the geometry read (from mu, scale, quat, opac, which may then be pinned host
// memory) is also written to the device arrays of copy.
template <int DEG, bool COLOR>
__global__ void __launch_bounds__(kProjWarps * 32) project_fwd_kernel(
    const float *__restrict__ mu, const float *__restrict__ scale, const float *__restrict__ quat,
    const float *__restrict__ opac, const float *__restrict__ sh, int64_t n, CamSet cs, XprConfig cfg,
    float *__restrict__ rec, int4 *__restrict__ bbox, int *__restrict__ tcount, int *__restrict__ isect_count,
    XprPrimsGrad copy) {
    grid_dep_wait();
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
    if (valid && copy.mu) {
        for (int j = 0; j < 3; ++j) {
            copy.mu[3 * i + j] = P.m[j];
            copy.scale[3 * i + j] = P.s[j];
        }
        reinterpret_cast<float4 *>(copy.quat)[i] = make_float4(P.q[0], P.q[1], P.q[2], P.q[3]);
        copy.opacity[i] = P.o;
    }
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
    grid_dep_wait();
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


// K6 for one view: chains d_rec = (d mu_2D, d conic, d o, d rgb) back to the parameters:
//   conic = A^{-1}:        dL/dA = -A^{-1} G A^{-1}  (G = dL/dconic, off-diagonal split in two)
//   A = T Sigma T^T + dI:   dL/dSigma = T^T dA T,  dL/dT = 2 dA T Sigma
//   T = J W:                dL/dJ = dL/dT W^T;  J(m_c) with the clamp (clamped coordinate is constant)
//   m_c = W mu + t;  mu_2D = (fx x/z + cx, fy y/z + cy)
//   Sigma = M M^T, M = R diag(s):  dL/dM = 2 dL/dSigma M
//   R(q/|q|):               explicit partials of the rotation matrix
//   colour:                 dL/dsh_k = Y_k g (where unclamped); dL/dd through the basis gradient,
//                           projected on the tangent plane and divided by |mu - camera centre|
// colour_adjoint with dL/dsh written instead of added; dsh may be the staged row shi itself (each
// coefficient's gradient is written after that coefficient's last read).
template <int DEG>
__device__ __forceinline__ void colour_adjoint_set(const Params &P, const float *shi, float *dsh, const Cam &k,
                                                   const float *drgb, float *gmu) {
    constexpr int K = (DEG + 1) * (DEG + 1);
    const float vx = P.m[0] - k.cpos[0], vy = P.m[1] - k.cpos[1], vz = P.m[2] - k.cpos[2];
    const float vinv = rsqrtf(vx * vx + vy * vy + vz * vz);
    const float ux = vx * vinv, uy = vy * vinv, uz = vz * vinv;
    float wk[K];
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
            dsh[3 * kk] = Y[kk] * gc[0];
            dsh[3 * kk + 1] = Y[kk] * gc[1];
            dsh[3 * kk + 2] = Y[kk] * gc[2];
        }
    }
    const float3 gdir = sh_grad_dot<DEG>(ux, uy, uz, wk);
    const float dd = gdir.x * ux + gdir.y * uy + gdir.z * uz;
    gmu[0] += (gdir.x - ux * dd) * vinv;
    gmu[1] += (gdir.y - uy * dd) * vinv;
    gmu[2] += (gdir.z - uz * dd) * vinv;
}

template <int DEG, bool SET = false>
__device__ __forceinline__ void adjoint_view(const Params &P, const float *shi, float *dsh, const Geo &G,
                                             const Cam &k, float4 d0, float4 d1, float4 d2, Acc<DEG> &A) {
    const float dmx = d0.x, dmy = d0.y, g00 = d0.z, g01 = d0.w, g11 = d1.x;
    const float drgb[3] = {d1.z, d1.w, d2.x};
    A.o += d1.y;

    if (SET)
        colour_adjoint_set<DEG>(P, shi, dsh, k, drgb, A.mu);
    else
        colour_adjoint<DEG>(P, shi, dsh, k, drgb, A.mu);

    // ---- mu_2D
    const float x = G.mc[0], y = G.mc[1], z = G.mc[2];
    const float iz = 1.f / z, iz2 = iz * iz;
    float gmc[3];
    gmc[0] = dmx * k.fx * iz;
    gmc[1] = dmy * k.fy * iz;
    gmc[2] = -(dmx * k.fx * x + dmy * k.fy * y) * iz2;
    gmc[2] += d2.y;  // rendered depth (record entry 9 = camera z)

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
    rotation_adjoint(G.qn, gR, A.qn);
}

// One thread per primitive; each warp stages its 32 primitives' SH coefficients in shared memory
// with coalesced 16-byte loads (all of a lane's loads issued before its first store) and
// accumulates their gradients there, then writes them out coalesced (a thread's own rows are 3K
// floats apart in global memory).  With one view the gradient overwrites the thread's own staged
// row after its last read, so a warp holds one row buffer (6.3 KB at degree 3) instead of two;
// with at most 96 registers, 5 blocks (20 warps) fit an SM.
template <int DEG>
__global__ void __launch_bounds__(kBwdWarps * 32, 5) project_bwd_kernel(
    const float *__restrict__ mu, const float *__restrict__ scale, const float *__restrict__ quat,
    const float *__restrict__ opac, const float *__restrict__ sh, int64_t n, CamSet cs, XprConfig cfg,
    const float *__restrict__ d_rec, float *__restrict__ gmu, float *__restrict__ gscale, float *__restrict__ gquat,
    float *__restrict__ gopac, float *__restrict__ gsh) {
    grid_dep_wait();
    constexpr int KC = (DEG + 1) * (DEG + 1) * 3;
    constexpr int LD = sh_ld<DEG>();
    extern __shared__ float s_bwd[];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t base = ((int64_t)blockIdx.x * kBwdWarps + w) * 32;
    if (base >= n) return;
    const int nv = (int)min((int64_t)32, n - base);
    const bool one = cs.n_views == 1;  // one row buffer: the gradient overwrites the staged row
    float *ssh = s_bwd + (size_t)w * (one ? 1 : 2) * 32 * LD;
    float *sdsh = one ? ssh : ssh + 32 * LD;
    const int64_t i = base + lane;
    Params P = {};
    if (i < n) P = load_params(mu, scale, quat, opac, i);
    stage_sh<DEG>(sh, base, nv, ssh);
    if (!one)
        for (int c = 0; c < KC; ++c) sdsh[lane * LD + c] = 0.f;
    __syncwarp();
    if (i < n) {
        Acc<DEG> A = {};
        float qinv = 0.f, qn[4] = {0.f, 0.f, 0.f, 0.f};
        bool wrote = false;  // one view: the row holds the SH gradient instead of the coefficients
        for (int v = 0; v < cs.n_views; ++v) {
            const Cam k = make_cam(cs.cam[v], cfg);
            Geo G;
            geometry(P, k, cfg.cov_dilation, G);
            if (!footprint(G, P.o, k, cfg).vis) continue;  // invisible in this view: no gradient from it
            const float4 *D4 = reinterpret_cast<const float4 *>(d_rec + ((size_t)v * n + i) * XPR_REC_FLOATS);
            if (one)
                adjoint_view<DEG, true>(P, ssh + lane * LD, sdsh + lane * LD, G, k, __ldg(D4), __ldg(D4 + 1),
                                        __ldg(D4 + 2), A);
            else
                adjoint_view<DEG>(P, ssh + lane * LD, sdsh + lane * LD, G, k, __ldg(D4), __ldg(D4 + 1), __ldg(D4 + 2),
                                  A);
            wrote = true;
            qinv = G.qinv;
            for (int j = 0; j < 4; ++j) qn[j] = G.qn[j];
        }
        if (one && !wrote)  // invisible: the staged coefficients become a zero gradient
            for (int c = 0; c < KC; ++c) sdsh[lane * LD + c] = 0.f;
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
    write_sh_rows<DEG>(sdsh, nv, gsh + base * KC);
}

// ---- multi-scene items: item k projects primitives [prim0, prim0 + n) of the concatenated arrays
// with camera k into its records [rec0, rec0 + n) (a block of whole warps: rec0 is a multiple of 32).
struct ItemSet {
    int count;
    int64_t rec0[kMaxItems + 1];  // first record of each item, then the total
    int64_t prim0[kMaxItems];
    int64_t n[kMaxItems];
    XprCamera cam[kMaxItems];
};

__device__ __forceinline__ int item_of_record(const ItemSet &is, int64_t r) {
    int k = 0;
#pragma unroll 1
    while (k + 1 < is.count && r >= is.rec0[k + 1]) ++k;
    return k;
}

template <int DEG>
__global__ void __launch_bounds__(kProjWarps * 32) project_items_kernel(
    const float *__restrict__ mu, const float *__restrict__ scale, const float *__restrict__ quat,
    const float *__restrict__ opac, const float *__restrict__ sh, ItemSet is, XprConfig cfg,
    float *__restrict__ rec, int4 *__restrict__ bbox, int *__restrict__ tcount, int *__restrict__ isect_count) {
    grid_dep_wait();
    constexpr int LD = sh_ld<DEG>();
    extern __shared__ float s_fwd[];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t base = ((int64_t)blockIdx.x * kProjWarps + w) * 32;  // first record of the warp
    if (base >= is.rec0[is.count]) return;
    const int k = item_of_record(is, base);  // warp-uniform: items start at multiples of 32
    const int64_t local = base - is.rec0[k];
    const int nv = (int)max((int64_t)0, min((int64_t)32, is.n[k] - local));
    const int64_t r = base + lane;
    const int64_t p0 = is.prim0[k] + local;
    float *ssh = s_fwd + (size_t)w * 32 * LD;
    if (nv > 0) stage_sh<DEG>(sh, p0, nv, ssh);
    CullData cd = {};
    int4 bb = make_int4(0, 0, 0, 0);
    int area = 0;
    if (lane < nv) {
        const Params P = load_params(mu, scale, quat, opac, p0 + lane);
        project_view<DEG>(P, ssh + lane * LD, r, is.cam[k], cfg, rec, bbox, tcount, cd, bb, area);
    } else {  // padding records of the item's block: invisible
        float4 *o4 = reinterpret_cast<float4 *>(rec + (size_t)r * XPR_REC_FLOATS);
        o4[0] = o4[1] = o4[2] = make_float4(0.f, 0.f, 0.f, 0.f);
        bbox[r] = make_int4(0, 0, 0, 0);
        tcount[r] = 0;
    }
    if (isect_count) {  // exact kept (primitive, tile) pairs with the binning's cull (warp-wide)
        const int cnt = count_kept_tiles(cd, bb, area, make_grid(is.cam[k], cfg));
        isect_count[r] = cnt;
    }
}

// Adjoint of the items' projection: each record's gradient is added (atomically: several items
// may view one scene) into its scene primitive's entries of the concatenated gradient arrays.
template <int DEG>
__global__ void __launch_bounds__(kBwdWarps * 32) project_bwd_items_kernel(
    const float *__restrict__ mu, const float *__restrict__ scale, const float *__restrict__ quat,
    const float *__restrict__ opac, const float *__restrict__ sh, ItemSet is, XprConfig cfg,
    const float *__restrict__ d_rec, float *__restrict__ gmu, float *__restrict__ gscale, float *__restrict__ gquat,
    float *__restrict__ gopac, float *__restrict__ gsh) {
    grid_dep_wait();
    constexpr int KC = (DEG + 1) * (DEG + 1) * 3;
    constexpr int LD = sh_ld<DEG>();
    extern __shared__ float s_bwd[];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t base = ((int64_t)blockIdx.x * kBwdWarps + w) * 32;
    if (base >= is.rec0[is.count]) return;
    const int k = item_of_record(is, base);
    const int64_t local = base - is.rec0[k];
    const int nv = (int)max((int64_t)0, min((int64_t)32, is.n[k] - local));
    if (nv == 0) return;
    const int64_t p0 = is.prim0[k] + local;
    float *ssh = s_bwd + (size_t)w * 2 * 32 * LD;
    float *sdsh = ssh + 32 * LD;
    stage_sh<DEG>(sh, p0, nv, ssh);
    for (int c = 0; c < KC; ++c) sdsh[lane * LD + c] = 0.f;
    __syncwarp();
    if (lane < nv) {
        const int64_t i = p0 + lane, r = base + lane;
        const Params P = load_params(mu, scale, quat, opac, i);
        const Cam kc = make_cam(is.cam[k], cfg);
        Geo G;
        geometry(P, kc, cfg.cov_dilation, G);
        if (footprint(G, P.o, kc, cfg).vis) {
            Acc<DEG> A = {};
            const float4 *D4 = reinterpret_cast<const float4 *>(d_rec + (size_t)r * XPR_REC_FLOATS);
            adjoint_view<DEG>(P, ssh + lane * LD, sdsh + lane * LD, G, kc, __ldg(D4), __ldg(D4 + 1), __ldg(D4 + 2), A);
            const float dot = A.qn[0] * G.qn[0] + A.qn[1] * G.qn[1] + A.qn[2] * G.qn[2] + A.qn[3] * G.qn[3];
            for (int j = 0; j < 3; ++j) {
                atomicAdd(gmu + 3 * i + j, A.mu[j]);
                atomicAdd(gscale + 3 * i + j, A.s[j]);
            }
            for (int j = 0; j < 4; ++j) atomicAdd(gquat + 4 * i + j, (A.qn[j] - G.qn[j] * dot) * G.qinv);
            atomicAdd(gopac + i, A.o);
        }
    }
    __syncwarp();
    float *go = gsh + p0 * KC;
    for (int e = lane; e < nv * KC; e += 32) {
        const int pi = e / KC;
        const float x = sdsh[pi * LD + (e - pi * KC)];
        if (x != 0.f) atomicAdd(go + e, x);
    }
}

ItemSet make_itemset(const XprCamera *cams, const XprItem *items, int n_items) {
    ItemSet is;
    memset(&is, 0, sizeof(is));
    is.count = n_items;
    for (int k = 0; k < n_items; ++k) {
        is.rec0[k] = items[k].rec_offset;
        is.prim0[k] = items[k].prim_offset;
        is.n[k] = items[k].n;
        is.cam[k] = cams[k];
    }
    is.rec0[n_items] = items[n_items - 1].rec_offset + (items[n_items - 1].n + 31) / 32 * 32;
    return is;
}

}  // namespace

int launch_project_items(const XprPrims &p, const XprCamera *cams, const XprItem *items, int n_items,
                         const XprConfig &cfg, float *rec, int32_t *bbox, int32_t *tc, cudaStream_t st,
                         int32_t *isect_count) {
    const ItemSet is = make_itemset(cams, items, n_items);
    const int64_t R = is.rec0[n_items];
    if (R == 0) return XPR_OK;
    const int tpb = kProjWarps * 32;
    const unsigned blocks = (unsigned)((R + tpb - 1) / tpb);
    XPR_DEG_DISPATCH(DEG, XPR_CUDA_TRY(launch_dependent(project_items_kernel<DEG>, dim3(blocks), dim3(tpb),
                                                        (size_t)kProjWarps * 32 * sh_ld<DEG>() * sizeof(float), st,
                                                        p.mu, p.scale, p.quat, p.opacity, p.sh, is, cfg, rec,
                                                        reinterpret_cast<int4 *>(bbox), tc, isect_count)));
    XPR_LAUNCH_CHECK("project_items_kernel");
    return XPR_OK;
}

int launch_project_bwd_items(const XprPrims &p, int64_t n_prims, const XprCamera *cams, const XprItem *items,
                             int n_items, const XprConfig &cfg, const float *d_rec, const XprPrimsGrad &g,
                             cudaStream_t st) {
    const int K = (cfg.sh_degree + 1) * (cfg.sh_degree + 1);
    XPR_CUDA_TRY(cudaMemsetAsync(g.mu, 0, (size_t)n_prims * 3 * sizeof(float), st));
    XPR_CUDA_TRY(cudaMemsetAsync(g.scale, 0, (size_t)n_prims * 3 * sizeof(float), st));
    XPR_CUDA_TRY(cudaMemsetAsync(g.quat, 0, (size_t)n_prims * 4 * sizeof(float), st));
    XPR_CUDA_TRY(cudaMemsetAsync(g.opacity, 0, (size_t)n_prims * sizeof(float), st));
    XPR_CUDA_TRY(cudaMemsetAsync(g.sh, 0, (size_t)n_prims * K * 3 * sizeof(float), st));
    const ItemSet is = make_itemset(cams, items, n_items);
    const int64_t R = is.rec0[n_items];
    if (R == 0) return XPR_OK;
    const int tpb = kBwdWarps * 32;
    const unsigned blocks = (unsigned)((R + tpb - 1) / tpb);
    cudaError_t attr = cudaSuccess;
    XPR_DEG_DISPATCH(DEG, {
        const size_t smem = (size_t)kBwdWarps * 2 * 32 * sh_ld<DEG>() * sizeof(float);
        attr = cudaFuncSetAttribute(project_bwd_items_kernel<DEG>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)smem);
        if (attr == cudaSuccess)
            XPR_CUDA_TRY(launch_dependent(project_bwd_items_kernel<DEG>, dim3(blocks), dim3(tpb), smem, st, p.mu,
                                          p.scale, p.quat, p.opacity, p.sh, is, cfg, d_rec, g.mu, g.scale, g.quat,
                                          g.opacity, g.sh));
    });
    XPR_CUDA_TRY(attr);
    XPR_LAUNCH_CHECK("project_bwd_items_kernel");
    return XPR_OK;
}

int launch_project_fwd_views(const XprPrims &p, int64_t n, const XprCamera *cams, int n_views, const XprConfig &cfg,
                             float *rec, int32_t *bbox, int32_t *tc, int32_t *isect_count, cudaStream_t st,
                             const XprPrimsGrad *copy) {
    if (n == 0 || n_views == 0) return XPR_OK;
    const XprPrimsGrad cp = copy ? *copy : XprPrimsGrad{nullptr, nullptr, nullptr, nullptr, nullptr};
    const int tpb = kProjWarps * 32;
    const unsigned blocks = (unsigned)((n + tpb - 1) / tpb);
    const CamSet cs = make_camset(cams, n_views);
    if (p.sh) {
        XPR_DEG_DISPATCH(DEG, XPR_CUDA_TRY(launch_dependent(project_fwd_kernel<DEG, true>, dim3(blocks), dim3(tpb),
                                                            (size_t)kProjWarps * 32 * sh_ld<DEG>() * sizeof(float), st,
                                                            p.mu, p.scale, p.quat, p.opacity, p.sh, n, cs, cfg, rec,
                                                            reinterpret_cast<int4 *>(bbox), tc, isect_count, cp)));
    } else {
        XPR_DEG_DISPATCH(DEG, XPR_CUDA_TRY(launch_dependent(project_fwd_kernel<DEG, false>, dim3(blocks), dim3(tpb), 0,
                                                            st, p.mu, p.scale, p.quat, p.opacity,
                                                            (const float *)nullptr, n, cs, cfg, rec,
                                                            reinterpret_cast<int4 *>(bbox), tc, isect_count, cp)));
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
    XPR_DEG_DISPATCH(DEG, XPR_CUDA_TRY(launch_dependent(project_color_kernel<DEG>, dim3(blocks), dim3(tpb),
                                                        (size_t)kProjWarps * 32 * sh_ld<DEG>() * sizeof(float), st, mu,
                                                        sh, n, cs, cfg, rec)));
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
        // one view: one row buffer per warp (half the limit)
        if (attr == cudaSuccess)
            attr = launch_dependent(project_bwd_kernel<DEG>, dim3(blocks), dim3(tpb), n_views == 1 ? smem / 2 : smem,
                                    st, p.mu, p.scale, p.quat, p.opacity, p.sh, n, cs, cfg, d_rec, g.mu, g.scale,
                                    g.quat, g.opacity, g.sh);
    });
    XPR_CUDA_TRY(attr);
    XPR_LAUNCH_CHECK("project_bwd_kernel");
    return XPR_OK;
}

int launch_project_fwd(const XprPrims &p, int64_t n, const XprCamera &cam, const XprConfig &cfg, float *rec,
                       int32_t *bbox, int32_t *tc, int32_t *isect_count, cudaStream_t st, const XprPrimsGrad *copy) {
    return launch_project_fwd_views(p, n, &cam, 1, cfg, rec, bbox, tc, isect_count, st, copy);
}

int launch_project_bwd(const XprPrims &p, int64_t n, const XprCamera &cam, const XprConfig &cfg,
                       const float *d_rec, const XprPrimsGrad &g, cudaStream_t st) {
    return launch_project_bwd_views(p, n, &cam, 1, cfg, d_rec, g, st);
}

}  // namespace xpr
