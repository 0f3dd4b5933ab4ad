// Preprocess stage: 3DGS projection (K1) and its adjoint (K6).
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
// One thread per primitive; the primitive SoA is read once and the 48-byte record is
// written with three float4 stores.
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

__device__ __forceinline__ void sh_basis(int deg, float x, float y, float z, float *Y) {
    Y[0] = kC0;
    if (deg < 1) return;
    Y[1] = -kC1 * y;
    Y[2] = kC1 * z;
    Y[3] = -kC1 * x;
    if (deg < 2) return;
    float xx = x * x, yy = y * y, zz = z * z;
    Y[4] = kC2a * x * y;
    Y[5] = -kC2a * y * z;
    Y[6] = kC2b * (2.f * zz - xx - yy);
    Y[7] = -kC2a * x * z;
    Y[8] = kC2c * (xx - yy);
    if (deg < 3) return;
    Y[9] = -kC3a * y * (3.f * xx - yy);
    Y[10] = kC3b * x * y * z;
    Y[11] = -kC3c * y * (4.f * zz - xx - yy);
    Y[12] = kC3d * z * (2.f * zz - 3.f * xx - 3.f * yy);
    Y[13] = -kC3c * x * (4.f * zz - xx - yy);
    Y[14] = kC3e * z * (xx - yy);
    Y[15] = -kC3a * x * (xx - 3.f * yy);
}

// Partial derivatives of the polynomials above w.r.t. (x, y, z); G[k] = (dYk/dx, dYk/dy, dYk/dz).
__device__ __forceinline__ void sh_basis_grad(int deg, float x, float y, float z, float3 *G) {
    G[0] = make_float3(0.f, 0.f, 0.f);
    if (deg < 1) return;
    G[1] = make_float3(0.f, -kC1, 0.f);
    G[2] = make_float3(0.f, 0.f, kC1);
    G[3] = make_float3(-kC1, 0.f, 0.f);
    if (deg < 2) return;
    float xx = x * x, yy = y * y, zz = z * z;
    G[4] = make_float3(kC2a * y, kC2a * x, 0.f);
    G[5] = make_float3(0.f, -kC2a * z, -kC2a * y);
    G[6] = make_float3(-2.f * kC2b * x, -2.f * kC2b * y, 4.f * kC2b * z);
    G[7] = make_float3(-kC2a * z, 0.f, -kC2a * x);
    G[8] = make_float3(2.f * kC2c * x, -2.f * kC2c * y, 0.f);
    if (deg < 3) return;
    G[9] = make_float3(-kC3a * 6.f * x * y, -kC3a * (3.f * xx - 3.f * yy), 0.f);
    G[10] = make_float3(kC3b * y * z, kC3b * x * z, kC3b * x * y);
    G[11] = make_float3(kC3c * 2.f * x * y, -kC3c * (4.f * zz - xx - 3.f * yy), -kC3c * 8.f * y * z);
    G[12] = make_float3(-kC3d * 6.f * x * z, -kC3d * 6.f * y * z, kC3d * (6.f * zz - 3.f * xx - 3.f * yy));
    G[13] = make_float3(-kC3c * (4.f * zz - 3.f * xx - yy), kC3c * 2.f * x * y, -kC3c * 8.f * x * z);
    G[14] = make_float3(kC3e * 2.f * x * z, -kC3e * 2.f * y * z, kC3e * (xx - yy));
    G[15] = make_float3(-kC3a * (3.f * xx - 3.f * yy), kC3a * 6.f * x * y, 0.f);
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

__device__ __forceinline__ void geometry(const float *mu, const float *s, const float *q, const Cam &k, float dil,
                                         Geo &G) {
    for (int i = 0; i < 3; ++i)
        G.mc[i] = k.W[3 * i] * mu[0] + k.W[3 * i + 1] * mu[1] + k.W[3 * i + 2] * mu[2] + k.t[i];
    float qq = q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3];
    G.qinv = rsqrtf(qq);
    for (int i = 0; i < 4; ++i) G.qn[i] = q[i] * G.qinv;
    quat_to_rot(G.qn[0], G.qn[1], G.qn[2], G.qn[3], G.R);
    float M[9];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) M[3 * i + j] = G.R[3 * i + j] * s[j];
    G.Sig[0] = M[0] * M[0] + M[1] * M[1] + M[2] * M[2];
    G.Sig[1] = M[0] * M[3] + M[1] * M[4] + M[2] * M[5];
    G.Sig[2] = M[0] * M[6] + M[1] * M[7] + M[2] * M[8];
    G.Sig[3] = M[3] * M[3] + M[4] * M[4] + M[5] * M[5];
    G.Sig[4] = M[3] * M[6] + M[4] * M[7] + M[5] * M[8];
    G.Sig[5] = M[6] * M[6] + M[7] * M[7] + M[8] * M[8];
    float x = G.mc[0], y = G.mc[1], z = G.mc[2];
    float iz = 1.f / z;
    float rx = x * iz, ry = y * iz;
    G.ux = fminf(fmaxf(rx, -k.limx), k.limx);
    G.uy = fminf(fmaxf(ry, -k.limy), k.limy);
    G.clx = (rx < -k.limx) || (rx > k.limx);
    G.cly = (ry < -k.limy) || (ry > k.limy);
    float J00 = k.fx * iz, J02 = -k.fx * G.ux * iz, J11 = k.fy * iz, J12 = -k.fy * G.uy * iz;
    for (int j = 0; j < 3; ++j) {
        G.T[j] = J00 * k.W[j] + J02 * k.W[6 + j];
        G.T[3 + j] = J11 * k.W[3 + j] + J12 * k.W[6 + j];
    }
    // Sigma_2D' = T Sigma T^T
    const float *T0 = G.T, *T1 = G.T + 3;
    const float *S = G.Sig;
    float u0[3] = {S[0] * T0[0] + S[1] * T0[1] + S[2] * T0[2], S[1] * T0[0] + S[3] * T0[1] + S[4] * T0[2],
                   S[2] * T0[0] + S[4] * T0[1] + S[5] * T0[2]};
    float u1[3] = {S[0] * T1[0] + S[1] * T1[1] + S[2] * T1[2], S[1] * T1[0] + S[3] * T1[1] + S[4] * T1[2],
                   S[2] * T1[0] + S[4] * T1[1] + S[5] * T1[2]};
    G.a = T0[0] * u0[0] + T0[1] * u0[1] + T0[2] * u0[2] + dil;
    G.b = T0[0] * u1[0] + T0[1] * u1[1] + T0[2] * u1[2];
    G.c = T1[0] * u1[0] + T1[1] * u1[1] + T1[2] * u1[2] + dil;
    G.det = G.a * G.c - G.b * G.b;
    G.mx = k.fx * rx + k.cx;
    G.my = k.fy * ry + k.cy;
}

__device__ __forceinline__ void project_one(const float *__restrict__ mu, const float *__restrict__ scale,
                                            const float *__restrict__ quat, const float *__restrict__ opac,
                                            const float *__restrict__ sh, int64_t i, const XprCamera &cam,
                                            const XprConfig &cfg, float *__restrict__ rec, int4 *__restrict__ bbox,
                                            int *__restrict__ tcount, CullData &cd, int4 &bb, int &area);

__global__ void __launch_bounds__(256) project_fwd_kernel(const float *__restrict__ mu, const float *__restrict__ scale,
                                                          const float *__restrict__ quat,
                                                          const float *__restrict__ opac,
                                                          const float *__restrict__ sh, int64_t n, XprCamera cam,
                                                          XprConfig cfg, float *__restrict__ rec,
                                                          int4 *__restrict__ bbox, int *__restrict__ tcount,
                                                          int *__restrict__ isect_count) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    CullData cd = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    int4 bb = make_int4(0, 0, 0, 0);
    int area = 0;
    if (i < n) project_one(mu, scale, quat, opac, sh, i, cam, cfg, rec, bbox, tcount, cd, bb, area);
    if (isect_count) {  // exact number of kept (primitive, tile) pairs, counted with the binning's cull
        const int cnt = count_kept_tiles(cd, bb, area, make_grid(cam, cfg));
        if (i < n) isect_count[i] = cnt;
    }
}

__device__ __forceinline__ void project_one(const float *__restrict__ mu, const float *__restrict__ scale,
                                            const float *__restrict__ quat, const float *__restrict__ opac,
                                            const float *__restrict__ sh, int64_t i, const XprCamera &cam,
                                            const XprConfig &cfg, float *__restrict__ rec, int4 *__restrict__ bbox,
                                            int *__restrict__ tcount, CullData &cd, int4 &bb, int &area) {
    const Cam k = make_cam(cam, cfg);
    const int deg = cfg.sh_degree;
    const int K = (deg + 1) * (deg + 1);
    float m[3] = {mu[3 * i], mu[3 * i + 1], mu[3 * i + 2]};
    float s[3] = {scale[3 * i], scale[3 * i + 1], scale[3 * i + 2]};
    float4 q4 = __ldg(reinterpret_cast<const float4 *>(quat) + i);
    float q[4] = {q4.x, q4.y, q4.z, q4.w};
    float o = opac[i];

    // colour
    float vx = m[0] - k.cpos[0], vy = m[1] - k.cpos[1], vz = m[2] - k.cpos[2];
    float vinv = rsqrtf(vx * vx + vy * vy + vz * vz);
    float Y[16];
    sh_basis(deg, vx * vinv, vy * vinv, vz * vinv, Y);
    float col[3] = {0.5f, 0.5f, 0.5f};
    const float *shi = sh + (size_t)i * K * 3;
    for (int kk = 0; kk < K; ++kk) {
        col[0] += shi[3 * kk] * Y[kk];
        col[1] += shi[3 * kk + 1] * Y[kk];
        col[2] += shi[3 * kk + 2] * Y[kk];
    }

    Geo G;
    geometry(m, s, q, k, cfg.cov_dilation, G);
    float z = G.mc[2];
    float4 *out = reinterpret_cast<float4 *>(rec + (size_t)i * XPR_REC_FLOATS);
    bool vis = (z > k.z_near) && (G.det > 0.f) && (o >= cfg.alpha_thresh);
    float lt = 0.f, ex = 0.f, ey = 0.f;
    int tc = 0;
    if (vis) {
        lt = logf(o / cfg.alpha_thresh);
        ex = sqrtf(2.f * lt * G.a);
        ey = sqrtf(2.f * lt * G.c);
        const float Wt = (float)((cam.width + cfg.tile_w - 1) / cfg.tile_w);
        const float Ht = (float)((cam.height + cfg.tile_h - 1) / cfg.tile_h);
        const float tw = (float)cfg.tile_w, th = (float)cfg.tile_h;
        bb.x = (int)fminf(fmaxf(floorf((G.mx - ex) / tw), 0.f), Wt);
        bb.y = (int)fminf(fmaxf(floorf((G.my - ey) / th), 0.f), Ht);
        bb.z = (int)fminf(fmaxf(floorf((G.mx + ex) / tw) + 1.f, 0.f), Wt);
        bb.w = (int)fminf(fmaxf(floorf((G.my + ey) / th) + 1.f, 0.f), Ht);
        tc = (bb.z - bb.x) * (bb.w - bb.y);
        vis = (fmaxf(ex, ey) > 0.f) && (tc > 0);
    }
    if (vis) {
        const float idet = 1.f / G.det;
        // the stored record values are the ones the cull reads back, so the count taken here from
        // registers and the emit kernel's decisions from memory are bit-identical
        cd.mx = G.mx;
        cd.my = G.my;
        cd.c0 = G.c * idet;
        cd.c1 = -G.b * idet;
        cd.c2 = G.a * idet;
        cd.lt = lt;
        cull_reciprocals(cd);
        out[0] = make_float4(cd.mx, cd.my, cd.c0, cd.c1);
        out[1] = make_float4(cd.c2, o, fmaxf(col[0], 0.f), fmaxf(col[1], 0.f));
        out[2] = make_float4(fmaxf(col[2], 0.f), z, lt, 1.f);
        bbox[i] = bb;
        tcount[i] = tc;
        area = tc;
    } else {
        out[0] = make_float4(0.f, 0.f, 0.f, 0.f);
        out[1] = make_float4(0.f, 0.f, 0.f, 0.f);
        out[2] = make_float4(0.f, z, 0.f, 0.f);
        bbox[i] = make_int4(0, 0, 0, 0);
        tcount[i] = 0;
        bb = make_int4(0, 0, 0, 0);
        area = 0;
    }
}

// K6: adjoint of the projection.  Recomputes the forward quantities, then chains
// d_rec = (d mu_2D, d conic, d o, d rgb) back to mu, scale, quat, opacity, sh:
//   conic = A^{-1}:        dL/dA = -A^{-1} G A^{-1}  (G = dL/dconic, off-diagonal split in two)
//   A = T Sigma T^T + dI:   dL/dSigma = T^T dA T,  dL/dT = 2 dA T Sigma
//   T = J W:                dL/dJ = dL/dT W^T;  J(m_c) with the clamp (clamped coordinate is constant)
//   m_c = W mu + t;  mu_2D = (fx x/z + cx, fy y/z + cy)
//   Sigma = M M^T, M = R diag(s):  dL/dM = 2 dL/dSigma M
//   R(q/|q|):               explicit partials of the rotation matrix, then the normalisation
//   colour:                 dL/dsh_k = Y_k g (where unclamped); dL/dd through the basis gradient,
//                           projected on the tangent plane and divided by |mu - camera centre|
__global__ void __launch_bounds__(256) project_bwd_kernel(const float *__restrict__ mu, const float *__restrict__ scale,
                                                          const float *__restrict__ quat,
                                                          const float *__restrict__ opac,
                                                          const float *__restrict__ sh, int64_t n, XprCamera cam,
                                                          XprConfig cfg, const float *__restrict__ d_rec,
                                                          float *__restrict__ gmu, float *__restrict__ gscale,
                                                          float *__restrict__ gquat, float *__restrict__ gopac,
                                                          float *__restrict__ gsh) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const Cam k = make_cam(cam, cfg);
    const int deg = cfg.sh_degree;
    const int K = (deg + 1) * (deg + 1);
    const float4 *D4 = reinterpret_cast<const float4 *>(d_rec + (size_t)i * XPR_REC_FLOATS);
    float4 d0 = __ldg(D4), d1 = __ldg(D4 + 1), d2 = __ldg(D4 + 2);
    float m[3] = {mu[3 * i], mu[3 * i + 1], mu[3 * i + 2]};
    float s[3] = {scale[3 * i], scale[3 * i + 1], scale[3 * i + 2]};
    float4 q4 = __ldg(reinterpret_cast<const float4 *>(quat) + i);
    float q[4] = {q4.x, q4.y, q4.z, q4.w};
    float o = opac[i];
    const float *shi = sh + (size_t)i * K * 3;
    float *gshi = gsh + (size_t)i * K * 3;

    Geo G;
    geometry(m, s, q, k, cfg.cov_dilation, G);
    bool vis = (G.mc[2] > k.z_near) && (G.det > 0.f) && (o >= cfg.alpha_thresh);
    if (vis) {
        // re-derive the bounding-box part of the visibility flag exactly as the forward does
        float lt = logf(o / cfg.alpha_thresh);
        float ex = sqrtf(2.f * lt * G.a), ey = sqrtf(2.f * lt * G.c);
        const float Wt = (float)((cam.width + cfg.tile_w - 1) / cfg.tile_w);
        const float Ht = (float)((cam.height + cfg.tile_h - 1) / cfg.tile_h);
        const float tw = (float)cfg.tile_w, th = (float)cfg.tile_h;
        int x0 = (int)fminf(fmaxf(floorf((G.mx - ex) / tw), 0.f), Wt);
        int y0 = (int)fminf(fmaxf(floorf((G.my - ey) / th), 0.f), Ht);
        int x1 = (int)fminf(fmaxf(floorf((G.mx + ex) / tw) + 1.f, 0.f), Wt);
        int y1 = (int)fminf(fmaxf(floorf((G.my + ey) / th) + 1.f, 0.f), Ht);
        vis = (fmaxf(ex, ey) > 0.f) && ((x1 - x0) * (y1 - y0) > 0);
    }
    if (!vis) {
        for (int j = 0; j < 3; ++j) {
            gmu[3 * i + j] = 0.f;
            gscale[3 * i + j] = 0.f;
        }
        reinterpret_cast<float4 *>(gquat)[i] = make_float4(0.f, 0.f, 0.f, 0.f);
        gopac[i] = 0.f;
        for (int e = 0; e < 3 * K; ++e) gshi[e] = 0.f;
        return;
    }
    const float dmx = d0.x, dmy = d0.y, g00 = d0.z, g01 = d0.w, g11 = d1.x;
    const float dop = d1.y;
    const float drgb[3] = {d1.z, d1.w, d2.x};

    // ---- colour
    float vx = m[0] - k.cpos[0], vy = m[1] - k.cpos[1], vz = m[2] - k.cpos[2];
    float vinv = rsqrtf(vx * vx + vy * vy + vz * vz);
    float dx_ = vx * vinv, dy_ = vy * vinv, dz_ = vz * vinv;
    float Y[16];
    float3 GY[16];
    sh_basis(deg, dx_, dy_, dz_, Y);
    sh_basis_grad(deg, dx_, dy_, dz_, GY);
    float raw[3] = {0.5f, 0.5f, 0.5f};
    for (int kk = 0; kk < K; ++kk) {
        raw[0] += shi[3 * kk] * Y[kk];
        raw[1] += shi[3 * kk + 1] * Y[kk];
        raw[2] += shi[3 * kk + 2] * Y[kk];
    }
    float gc[3];
    for (int c = 0; c < 3; ++c) gc[c] = raw[c] > 0.f ? drgb[c] : 0.f;
    float3 gdir = make_float3(0.f, 0.f, 0.f);
    for (int kk = 0; kk < K; ++kk) {
        float w = gc[0] * shi[3 * kk] + gc[1] * shi[3 * kk + 1] + gc[2] * shi[3 * kk + 2];
        gdir.x += w * GY[kk].x;
        gdir.y += w * GY[kk].y;
        gdir.z += w * GY[kk].z;
        gshi[3 * kk] = Y[kk] * gc[0];
        gshi[3 * kk + 1] = Y[kk] * gc[1];
        gshi[3 * kk + 2] = Y[kk] * gc[2];
    }
    float dd = gdir.x * dx_ + gdir.y * dy_ + gdir.z * dz_;
    float gm[3] = {(gdir.x - dx_ * dd) * vinv, (gdir.y - dy_ * dd) * vinv, (gdir.z - dz_ * dd) * vinv};

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
        // dSigma_ij = ga T0i T0j + gb (T0i T1j + T1i T0j) + gc T1i T1j
        int idx = 0;
        for (int a_ = 0; a_ < 3; ++a_)
            for (int b_ = a_; b_ < 3; ++b_) {
                gS[idx++] = ga * T0[a_] * T0[b_] + gb * (T0[a_] * T1[b_] + T1[a_] * T0[b_]) + gcv * T1[a_] * T1[b_];
            }
    }
    // T Sigma rows
    float TS0[3] = {T0[0] * S[0] + T0[1] * S[1] + T0[2] * S[2], T0[0] * S[1] + T0[1] * S[3] + T0[2] * S[4],
                    T0[0] * S[2] + T0[1] * S[4] + T0[2] * S[5]};
    float TS1[3] = {T1[0] * S[0] + T1[1] * S[1] + T1[2] * S[2], T1[0] * S[1] + T1[1] * S[3] + T1[2] * S[4],
                    T1[0] * S[2] + T1[1] * S[4] + T1[2] * S[5]};
    float gT0[3], gT1[3];
    for (int j = 0; j < 3; ++j) {
        gT0[j] = 2.f * (ga * TS0[j] + gb * TS1[j]);
        gT1[j] = 2.f * (gb * TS0[j] + gcv * TS1[j]);
    }
    // T = J W: dJ_rk = sum_b dT_rb W_kb ; only J00, J02, J11, J12 are non-zero
    const float *W = k.W;
    float gJ00 = gT0[0] * W[0] + gT0[1] * W[1] + gT0[2] * W[2];
    float gJ02 = gT0[0] * W[6] + gT0[1] * W[7] + gT0[2] * W[8];
    float gJ11 = gT1[0] * W[3] + gT1[1] * W[4] + gT1[2] * W[5];
    float gJ12 = gT1[0] * W[6] + gT1[1] * W[7] + gT1[2] * W[8];
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
    for (int j = 0; j < 3; ++j) gm[j] += W[j] * gmc[0] + W[3 + j] * gmc[1] + W[6 + j] * gmc[2];

    // ---- Sigma = M M^T, M = R diag(s): dM = 2 dSigma M
    float gSf[9] = {gS[0], gS[1], gS[2], gS[1], gS[3], gS[4], gS[2], gS[4], gS[5]};
    float M[9];
    for (int a_ = 0; a_ < 3; ++a_)
        for (int c_ = 0; c_ < 3; ++c_) M[3 * a_ + c_] = G.R[3 * a_ + c_] * s[c_];
    float gR[9];
    float gs[3] = {0.f, 0.f, 0.f};
    for (int a_ = 0; a_ < 3; ++a_)
        for (int c_ = 0; c_ < 3; ++c_) {
            float gM = 2.f * (gSf[3 * a_] * M[c_] + gSf[3 * a_ + 1] * M[3 + c_] + gSf[3 * a_ + 2] * M[6 + c_]);
            gs[c_] += gM * G.R[3 * a_ + c_];
            gR[3 * a_ + c_] = gM * s[c_];
        }
    // ---- R(qn): partials of the unit-quaternion rotation matrix
    const float w = G.qn[0], qx = G.qn[1], qy = G.qn[2], qz = G.qn[3];
    float gw = 2.f * (-qz * gR[1] + qy * gR[2] + qz * gR[3] - qx * gR[5] - qy * gR[6] + qx * gR[7]);
    float gx = 2.f * (qy * gR[1] + qz * gR[2] + qy * gR[3] - 2.f * qx * gR[4] - w * gR[5] + qz * gR[6] + w * gR[7] -
                      2.f * qx * gR[8]);
    float gy = 2.f * (-2.f * qy * gR[0] + qx * gR[1] + w * gR[2] + qx * gR[3] + qz * gR[5] - w * gR[6] + qz * gR[7] -
                      2.f * qy * gR[8]);
    float gz = 2.f * (-2.f * qz * gR[0] - w * gR[1] + qx * gR[2] + w * gR[3] - 2.f * qz * gR[4] + qy * gR[5] +
                      qx * gR[6] + qy * gR[7]);
    float dot = gw * w + gx * qx + gy * qy + gz * qz;
    float4 gq = make_float4((gw - w * dot) * G.qinv, (gx - qx * dot) * G.qinv, (gy - qy * dot) * G.qinv,
                            (gz - qz * dot) * G.qinv);

    for (int j = 0; j < 3; ++j) {
        gmu[3 * i + j] = gm[j];
        gscale[3 * i + j] = gs[j];
    }
    reinterpret_cast<float4 *>(gquat)[i] = gq;
    gopac[i] = dop;
}

}  // namespace

int launch_project_fwd(const XprPrims &p, int64_t n, const XprCamera &cam, const XprConfig &cfg, float *rec,
                       int32_t *bbox, int32_t *tc, int32_t *isect_count, cudaStream_t st) {
    if (n == 0) return XPR_OK;
    const int tpb = 256;
    const int64_t blocks = (n + tpb - 1) / tpb;
    project_fwd_kernel<<<(unsigned)blocks, tpb, 0, st>>>(p.mu, p.scale, p.quat, p.opacity, p.sh, n, cam, cfg, rec,
                                                         reinterpret_cast<int4 *>(bbox), tc, isect_count);
    XPR_LAUNCH_CHECK("project_fwd_kernel");
    return XPR_OK;
}

int launch_project_bwd(const XprPrims &p, int64_t n, const XprCamera &cam, const XprConfig &cfg,
                       const float *d_rec, const XprPrimsGrad &g, cudaStream_t st) {
    if (n == 0) return XPR_OK;
    const int tpb = 256;
    const int64_t blocks = (n + tpb - 1) / tpb;
    project_bwd_kernel<<<(unsigned)blocks, tpb, 0, st>>>(p.mu, p.scale, p.quat, p.opacity, p.sh, n, cam, cfg, d_rec,
                                                         g.mu, g.scale, g.quat, g.opacity, g.sh);
    XPR_LAUNCH_CHECK("project_bwd_kernel");
    return XPR_OK;
}

}  // namespace xpr
