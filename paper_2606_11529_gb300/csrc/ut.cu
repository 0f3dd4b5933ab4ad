// 3DGUT (Sec. 3 method examples; Appendix, implementation of XPR-3DGUT): unscented-transform
// projection, ray-evaluated compositing, and their adjoints.  The rest of the pipeline (depth
// order, binning with the ray-offset tile cull of cull.cuh, sort) is the 3DGS one, unchanged.
//
// Projection (per primitive and view):
//   seven sigma points X_0 = mu, X_{a,+-} = mu +- sqrt(3) s_a R e_a (UT with alpha = 1, beta = 2,
//   kappa = 0: mean weights 0 and 1/6, covariance weights 2 and 1/6), each through the pinhole
//   projection; mu_2D and Sigma_2D from the weighted points; low-pass dilation Sigma_2D + d I; the
//   Mip-Splatting opacity o' = o sqrt(det_0 / det); conic, extents and the tile box from mu_2D - 0.5
//   (pixel centres at +0.5).  A primitive is invisible when a sigma point lies at or behind the
//   near plane, det <= 0 or o' <= alpha_t.  The record rec[12] keeps the 3DGS layout (UT mean and
//   conic, o', rgb, depth, ln(o'/alpha_t), visible), so binning and sorting read it unchanged.
//   The sigma points enter only through their offsets from the projected centre p_0,
//     Delta_{a,+-} = +- f (D_a,x z_0 - x_0 D_a,z) / (z_{a,+-} z_0)   (D_a = W (sqrt(3) s_a R e_a)),
//   so Sigma_2D is formed from small differences computed without cancellation.
//
// Evaluation (per pixel and list entry): the paper writes the largest response along the pixel
// ray as exp(-|o_c + tau_max d_c|^2 / 2) with o_c = M (c - mu), d_c = M d, M = S^-1 R^T.  In
// float32 that form cancels: |o_c|^2 ~ (z / s)^2 is 10^4 .. 10^6 while the result is O(1).  The
// kernels evaluate the same minimum in the camera frame relative to the projected centre: with
// pixel offset (dx, dy) = (x + 0.5, y + 0.5) - p_0, the ray meets the depth plane of the mean at
// a point offset delta = (z_0 dx / fx, z_0 dy / fy, 0) from it, so in canonical coordinates
//   a = M W^T delta = dx A_0 + dy A_1,   A_0 = (z_0 / fx) M W^T e_0,  A_1 = (z_0 / fy) M W^T e_1,
// and the ray direction is b = a - o_c; the minimum over the line is
//   Q = |a|^2 - (a.b)^2 / |b|^2 = |e|^2,  e = a - kappa b,  kappa = a.b / |b|^2,
// with a.b = |a|^2 - a.o_c and |b|^2 = |a|^2 - 2 a.o_c + |o_c|^2.  G = exp(-Q / 2); valid iff
// G > 0.0113; alpha = min(alpha_max, o' G).  Shader data sd[16] per primitive:
//   [p0x p0y A0x A0y] [A0z A1x A1y A1z] [o_c (3) o'] [r g b |o_c|^2]
//
// Adjoint of the evaluation: dQ = -alpha dL/dalpha / 2 (unclamped), dL/da = 2 (1 - kappa) dQ e,
// dL/do_c = 2 kappa dQ e (|o_c|^2 folded in), then dA_0 = sum dL/da dx, dA_1 = sum dL/da dy,
// dp_0 = -(sum dL/da) . (A_0, A_1).  The projection adjoint chains (p_0, A_0, A_1, o_c, o', rgb)
// back to (mu, scale, quat, opacity, sh), the Mip-Splatting factor through the unscented
// covariance of the sigma points included.
#include "project_common.cuh"

namespace xpr {
namespace {

constexpr float kSqrt3 = 1.7320508075688772f;
constexpr float kUtValid = 0.0113f;  // validity threshold of the ray response

// Fisheye camera (equidistant projection with a radial polynomial): a camera-space point at angle
// theta = atan2(r, z) from the axis, r = |(x, y)|, lands at (fx s x + cx, fy s y + cy) with
// s = theta_d / r, theta_d = theta (1 + k1 theta^2 + k2 theta^4 + k3 theta^6 + k4 theta^8).
__device__ __forceinline__ float fish_thetad(const float *kk, float th) {
    const float t2 = th * th;
    return th * (1.f + t2 * (kk[0] + t2 * (kk[1] + t2 * (kk[2] + t2 * kk[3]))));
}
__device__ __forceinline__ float fish_thetad_prime(const float *kk, float th) {
    const float t2 = th * th;
    return 1.f + t2 * (3.f * kk[0] + t2 * (5.f * kk[1] + t2 * (7.f * kk[2] + t2 * 9.f * kk[3])));
}

// projection of a camera-space point to pixels (pinhole or fisheye)
__device__ __forceinline__ void cam_project(const Cam &k, float x, float y, float z, float &u, float &v) {
    if (k.model == 1) {
        const float r = sqrtf(x * x + y * y);
        const float s = r > 0.f ? fish_thetad(k.k, atan2f(r, z)) / r : 1.f / z;
        u = k.fx * s * x + k.cx;
        v = k.fy * s * y + k.cy;
    } else {
        u = k.fx * (x / z) + k.cx;
        v = k.fy * (y / z) + k.cy;
    }
}

// d(u, v)/d(x, y, z), 2x3 row-major.  Fisheye, with s = theta_d / r, t = theta_d' / (r^2 + z^2),
// K = (t z - s) / r^2: du/dx = fx (s + x^2 K), du/dy = fx x y K, du/dz = -fx x t, and v alike
// (on the axis s -> 1/z, t -> 1/z^2, K -> 2 (k1 - 1/3) / z^3).
__device__ __forceinline__ void cam_jacobian(const Cam &k, float x, float y, float z, float *J) {
    if (k.model != 1) {
        const float iz = 1.f / z;
        J[0] = k.fx * iz;
        J[1] = 0.f;
        J[2] = -k.fx * x * iz * iz;
        J[3] = 0.f;
        J[4] = k.fy * iz;
        J[5] = -k.fy * y * iz * iz;
        return;
    }
    const float r2 = x * x + y * y, r = sqrtf(r2);
    float s, t, K;
    if (r < 1e-6f * fabsf(z)) {
        s = 1.f / z;
        t = s * s;
        K = 2.f * (k.k[0] - 1.f / 3.f) * s * s * s;
    } else {
        const float th = atan2f(r, z);
        s = fish_thetad(k.k, th) / r;
        t = fish_thetad_prime(k.k, th) / (r2 + z * z);
        K = (t * z - s) / r2;
    }
    J[0] = k.fx * (s + x * x * K);
    J[1] = k.fx * x * y * K;
    J[2] = -k.fx * x * t;
    J[3] = k.fy * x * y * K;
    J[4] = k.fy * (s + y * y * K);
    J[5] = -k.fy * y * t;
}

// Forward quantities of the unscented projection (recomputed by the adjoint).
struct UtGeo {
    float qn[4], qinv;
    float R[9];
    float mc[3];     // camera-space mean (x_0, y_0, z_0)
    float WR[9];     // W R: column a is the camera-space direction of the sigma axis a
    float D[3][3];   // D[a] = sqrt(3) s_a WR e_a, camera-space sigma-point displacement
    float dl[6][2];  // Delta_k, k = 2a + (0: +, 1: -), pixel offsets of the sigma points from p_0
    float mo[2];     // mean offset mu_2D - p_0
    float c0, c1, c2;  // Sigma_2D before dilation
    float det0, det, mip;
    float M[9];      // S^-1 R^T
    float Mc[9];     // M W^T (canonical from camera coordinates)
    bool front;      // every sigma point in front of the near plane
};

__device__ __forceinline__ void ut_geometry(const Params &P, const Cam &k, float dil, UtGeo &U) {
    const float qq = P.q[0] * P.q[0] + P.q[1] * P.q[1] + P.q[2] * P.q[2] + P.q[3] * P.q[3];
    U.qinv = rsqrtf(qq);
    for (int i = 0; i < 4; ++i) U.qn[i] = P.q[i] * U.qinv;
    quat_to_rot(U.qn[0], U.qn[1], U.qn[2], U.qn[3], U.R);
    cam_point(k, P.m, U.mc);
    for (int i = 0; i < 3; ++i)
        for (int a = 0; a < 3; ++a)
            U.WR[3 * i + a] = k.W[3 * i] * U.R[a] + k.W[3 * i + 1] * U.R[3 + a] + k.W[3 * i + 2] * U.R[6 + a];
    for (int i = 0; i < 3; ++i) {
        const float is = 1.f / P.s[i];
        for (int j = 0; j < 3; ++j) U.M[3 * i + j] = U.R[3 * j + i] * is;
    }
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
            U.Mc[3 * i + j] = U.M[3 * i] * k.W[3 * j] + U.M[3 * i + 1] * k.W[3 * j + 1] + U.M[3 * i + 2] * k.W[3 * j + 2];
    const float x0 = U.mc[0], y0 = U.mc[1], z0 = U.mc[2];
    U.front = z0 > k.z_near;
    float sx = 0.f, sy = 0.f;
    float u0 = 0.f, v0 = 0.f;
    if (k.model == 1) cam_project(k, x0, y0, z0, u0, v0);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const float h = kSqrt3 * P.s[a];
        for (int i = 0; i < 3; ++i) U.D[a][i] = h * U.WR[3 * i + a];
        const float nx = U.D[a][0] * z0 - x0 * U.D[a][2];
        const float ny = U.D[a][1] * z0 - y0 * U.D[a][2];
#pragma unroll
        for (int e = 0; e < 2; ++e) {
            const float sg = e == 0 ? 1.f : -1.f;
            const float zk = z0 + sg * U.D[a][2];
            U.front = U.front && (zk > k.z_near);
            if (k.model == 1) {  // fisheye: difference of the projections
                float uk, vk;
                cam_project(k, x0 + sg * U.D[a][0], y0 + sg * U.D[a][1], zk, uk, vk);
                U.dl[2 * a + e][0] = uk - u0;
                U.dl[2 * a + e][1] = vk - v0;
            } else {  // pinhole: the offset in closed form, without cancellation
                const float f = sg / (zk * z0);
                U.dl[2 * a + e][0] = k.fx * nx * f;
                U.dl[2 * a + e][1] = k.fy * ny * f;
            }
            sx += U.dl[2 * a + e][0];
            sy += U.dl[2 * a + e][1];
        }
    }
    U.mo[0] = sx * (1.f / 6.f);
    U.mo[1] = sy * (1.f / 6.f);
    // centre point (offset 0, covariance weight 2) and the six others (weight 1/6)
    float c0 = 0.f, c1 = 0.f, c2 = 0.f;
#pragma unroll
    for (int kk = 0; kk < 6; ++kk) {
        const float dx = U.dl[kk][0] - U.mo[0], dy = U.dl[kk][1] - U.mo[1];
        c0 += dx * dx;
        c1 += dx * dy;
        c2 += dy * dy;
    }
    U.c0 = 2.f * U.mo[0] * U.mo[0] + c0 * (1.f / 6.f);
    U.c1 = 2.f * U.mo[0] * U.mo[1] + c1 * (1.f / 6.f);
    U.c2 = 2.f * U.mo[1] * U.mo[1] + c2 * (1.f / 6.f);
    U.det0 = U.c0 * U.c2 - U.c1 * U.c1;
    U.det = (U.c0 + dil) * (U.c2 + dil) - U.c1 * U.c1;
    U.mip = U.det > 0.f ? sqrtf(fmaxf(U.det0, 0.f) / U.det) : 0.f;
}

struct UtFootprint {
    bool vis;
    float o, lt, mx, my, ca, cb, cc;  // o', ln(o'/a_t), mu_2D, conic
    int4 bb;
    int tc;
};

__device__ __forceinline__ UtFootprint ut_footprint(const UtGeo &U, float o, const Cam &k, const XprConfig &cfg) {
    UtFootprint f = {};
    f.o = o * U.mip;
    f.vis = U.front && (U.det > 0.f) && (f.o > cfg.alpha_thresh);
    if (!f.vis) return f;
    const float a = U.c0 + cfg.cov_dilation, c = U.c2 + cfg.cov_dilation;
    const float idet = 1.f / U.det;
    f.ca = c * idet;
    f.cb = -U.c1 * idet;
    f.cc = a * idet;
    f.lt = logf(f.o / cfg.alpha_thresh);
    const float ex = sqrtf(2.f * f.lt * a), ey = sqrtf(2.f * f.lt * c);
    float u0, v0;
    cam_project(k, U.mc[0], U.mc[1], U.mc[2], u0, v0);
    f.mx = u0 + U.mo[0];
    f.my = v0 + U.mo[1];
    const float Wt = (float)((k.width + cfg.tile_w - 1) / cfg.tile_w);
    const float Ht = (float)((k.height + cfg.tile_h - 1) / cfg.tile_h);
    const float tw = (float)cfg.tile_w, th = (float)cfg.tile_h;
    const float bx = f.mx - 0.5f, by = f.my - 0.5f;  // ray offset: pixel centres at +0.5
    f.bb.x = (int)fminf(fmaxf(floorf((bx - ex) / tw), 0.f), Wt);
    f.bb.y = (int)fminf(fmaxf(floorf((by - ey) / th), 0.f), Ht);
    f.bb.z = (int)fminf(fmaxf(floorf((bx + ex) / tw) + 1.f, 0.f), Wt);
    f.bb.w = (int)fminf(fmaxf(floorf((by + ey) / th) + 1.f, 0.f), Ht);
    f.tc = (f.bb.z - f.bb.x) * (f.bb.w - f.bb.y);
    f.vis = (fmaxf(ex, ey) > 0.f) && (f.tc > 0);
    return f;
}

// One view of the unscented projection: writes rec / sd / bbox / tile count of record `out`.
template <int DEG>
__device__ __forceinline__ void ut_project_view(const Params &P, const float *shi, int64_t out, const XprCamera &cam,
                                                const XprConfig &cfg, float *__restrict__ rec,
                                                float *__restrict__ sd, int4 *__restrict__ bbox,
                                                int *__restrict__ tcount, CullData &cd, int4 &bb, int &area) {
    const Cam k = make_cam(cam, cfg);
    UtGeo U;
    ut_geometry(P, k, cfg.cov_dilation, U);
    const UtFootprint f = ut_footprint(U, P.o, k, cfg);
    float4 *o4 = reinterpret_cast<float4 *>(rec + (size_t)out * XPR_REC_FLOATS);
    float4 *s4 = reinterpret_cast<float4 *>(sd + (size_t)out * XPR_SD_FLOATS);
    if (!f.vis) {
        const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
        o4[0] = z4;
        o4[1] = z4;
        o4[2] = make_float4(0.f, U.mc[2], 0.f, 0.f);
        s4[0] = z4;
        s4[1] = z4;
        s4[2] = z4;
        s4[3] = z4;
        bbox[out] = make_int4(0, 0, 0, 0);
        tcount[out] = 0;
        bb = make_int4(0, 0, 0, 0);
        area = 0;
        return;
    }
    float col[3];
    sh_colour<DEG>(P, shi, k, col);
    for (int c = 0; c < 3; ++c) col[c] = fmaxf(col[c], 0.f);
    // the cull reads the stored record back, so count it from the same float values
    cd = make_cull(f.mx, f.my, f.ca, f.cb, f.cc, f.lt);
    o4[0] = make_float4(f.mx, f.my, f.ca, f.cb);
    o4[1] = make_float4(f.cc, f.o, col[0], col[1]);
    o4[2] = make_float4(col[2], U.mc[2], f.lt, 1.f);
    // shader data
    // the centre and the canonical images of the pixel axes: in pixels for the pinhole, in normalised
    // image coordinates (x/z, y/z) for the fisheye, whose pixel rays the render unprojects
    const float z0 = U.mc[2];
    const bool fish = k.model == 1;
    const float p0x = fish ? U.mc[0] / z0 : k.fx * (U.mc[0] / z0) + k.cx;
    const float p0y = fish ? U.mc[1] / z0 : k.fy * (U.mc[1] / z0) + k.cy;
    const float s0 = fish ? z0 : z0 / k.fx, s1 = fish ? z0 : z0 / k.fy;
    const float vx = k.cpos[0] - P.m[0], vy = k.cpos[1] - P.m[1], vz = k.cpos[2] - P.m[2];
    float roc[3];
    for (int i = 0; i < 3; ++i) roc[i] = U.M[3 * i] * vx + U.M[3 * i + 1] * vy + U.M[3 * i + 2] * vz;
    const float rr = roc[0] * roc[0] + roc[1] * roc[1] + roc[2] * roc[2];
    s4[0] = make_float4(p0x, p0y, s0 * U.Mc[0], s0 * U.Mc[3]);
    s4[1] = make_float4(s0 * U.Mc[6], s1 * U.Mc[1], s1 * U.Mc[4], s1 * U.Mc[7]);
    s4[2] = make_float4(roc[0], roc[1], roc[2], f.o);
    s4[3] = make_float4(col[0], col[1], col[2], rr);
    bbox[out] = f.bb;
    tcount[out] = f.tc;
    bb = f.bb;
    area = f.tc;
}

template <int DEG>
__global__ void __launch_bounds__(kProjWarps * 32) ut_project_fwd_kernel(
    const float *__restrict__ mu, const float *__restrict__ scale, const float *__restrict__ quat,
    const float *__restrict__ opac, const float *__restrict__ sh, int64_t n, CamSet cs, XprConfig cfg,
    float *__restrict__ rec, float *__restrict__ sd, int4 *__restrict__ bbox, int *__restrict__ tcount,
    int *__restrict__ isect_count) {
    grid_dep_wait();
    constexpr int LD = sh_ld<DEG>();
    extern __shared__ float s_utf[];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t base = ((int64_t)blockIdx.x * kProjWarps + w) * 32;
    if (base >= n) return;
    const int nv = (int)min((int64_t)32, n - base);
    float *ssh = s_utf + (size_t)w * 32 * LD;
    stage_sh<DEG>(sh, base, nv, ssh);
    const int64_t i = base + lane;
    const bool valid = i < n;
    Params P = {};
    if (valid) P = load_params(mu, scale, quat, opac, i);
    for (int v = 0; v < cs.n_views; ++v) {
        CullData cd = {};
        int4 bb = make_int4(0, 0, 0, 0);
        int area = 0;
        const int64_t out = (int64_t)v * n + i;
        if (valid) ut_project_view<DEG>(P, ssh + lane * LD, out, cs.cam[v], cfg, rec, sd, bbox, tcount, cd, bb, area);
        if (isect_count) {
            const int cnt = count_kept_tiles(cd, bb, area, make_grid(cs.cam[v], cfg));
            if (valid) isect_count[out] = cnt;
        }
    }
}

// Adjoint of one view of the unscented projection, from d_sd = (dp_0, dA_0, dA_1, do_c, do', drgb)
// to the parameters (accumulated in A and dsh):
//   p_0 = (fx x_0 / z_0 + cx, fy y_0 / z_0 + cy);  A_0 = (z_0 / fx) Mc e_0, A_1 = (z_0 / fy) Mc e_1;
//   Mc = M W^T;  o_c = M (c - mu);  M_ij = R_ji / s_i;  o' = o m, m = sqrt(det_0 / det) with
//   det_0 = c0 c2 - c1^2, det = (c0 + d)(c2 + d) - c1^2 and Sigma_2D = sum_k wc_k (Delta_k - mo)
//   (Delta_k - mo)^T, mo = sum_k wm_k Delta_k, Delta_k = proj(m_c + sg D_a) - proj(m_c),
//   D_a = sqrt(3) s_a W R e_a;  m_c = W mu + t;  colour as in 3DGS.
template <int DEG>
__device__ __forceinline__ void ut_adjoint_view(const Params &P, const float *shi, float *dsh, const UtGeo &U,
                                                const Cam &k, float dil, const float4 *d4, Acc<DEG> &A) {
    const float4 d0 = __ldg(d4), d1 = __ldg(d4 + 1), d2 = __ldg(d4 + 2), d3 = __ldg(d4 + 3);
    const float dp0x = d0.x, dp0y = d0.y;
    const float dA0[3] = {d0.z, d0.w, d1.x}, dA1[3] = {d1.y, d1.z, d1.w};
    const float droc[3] = {d2.x, d2.y, d2.z};
    const float dop = d2.w;
    const float drgb[3] = {d3.x, d3.y, d3.z};

    colour_adjoint<DEG>(P, shi, dsh, k, drgb, A.mu);
    A.o += dop * U.mip;
    const float gmip = dop * P.o;

    const float x0 = U.mc[0], y0 = U.mc[1], z0 = U.mc[2];
    const float iz = 1.f / z0, iz2 = iz * iz;
    // the shader data's units: pixels (pinhole, scale f) or normalised coordinates (fisheye, scale 1)
    const float fx = k.model == 1 ? 1.f : k.fx, fy = k.model == 1 ? 1.f : k.fy;
    float gmc[3];
    // p_0 = (fx x/z, fy y/z) (+ principal point)
    gmc[0] = dp0x * fx * iz;
    gmc[1] = dp0y * fy * iz;
    gmc[2] = -(dp0x * fx * x0 + dp0y * fy * y0) * iz2;
    // A_0 = (z / fx) Mc e_0, A_1 = (z / fy) Mc e_1
    const float s0 = z0 / fx, s1 = z0 / fy;
    gmc[2] += (dA0[0] * U.Mc[0] + dA0[1] * U.Mc[3] + dA0[2] * U.Mc[6]) / fx +
              (dA1[0] * U.Mc[1] + dA1[1] * U.Mc[4] + dA1[2] * U.Mc[7]) / fy;
    // Mc = M W^T (columns 0 and 1 only): dM_ik = sum_j dMc_ij W_jk; plus o_c = M (c - mu)
    const float v[3] = {k.cpos[0] - P.m[0], k.cpos[1] - P.m[1], k.cpos[2] - P.m[2]};
    float gM[9];
    for (int i = 0; i < 3; ++i)
        for (int kk = 0; kk < 3; ++kk)
            gM[3 * i + kk] = s0 * dA0[i] * k.W[kk] + s1 * dA1[i] * k.W[3 + kk] + droc[i] * v[kk];
    for (int kk = 0; kk < 3; ++kk) A.mu[kk] -= U.M[kk] * droc[0] + U.M[3 + kk] * droc[1] + U.M[6 + kk] * droc[2];
    // M_ij = R_ji / s_i
    float gR[9];
    for (int i = 0; i < 3; ++i) {
        const float is = 1.f / P.s[i];
        float acc = 0.f;
        for (int j = 0; j < 3; ++j) {
            acc += gM[3 * i + j] * U.M[3 * i + j];
            gR[3 * j + i] = gM[3 * i + j] * is;
        }
        A.s[i] -= acc * is;
    }
    // Mip-Splatting factor through the unscented covariance
    if (gmip != 0.f && U.det0 > 0.f) {
        const float kd0 = gmip * U.mip / (2.f * U.det0), kd = -gmip * U.mip / (2.f * U.det);
        const float gc0 = kd0 * U.c2 + kd * (U.c2 + dil);
        const float gc2 = kd0 * U.c0 + kd * (U.c0 + dil);
        const float gc1 = -2.f * U.c1 * (kd0 + kd);
        // centre point: Delta_0 = 0, weight 2
        float gmx = -2.f * (2.f * gc0 * -U.mo[0] + gc1 * -U.mo[1]);
        float gmy = -2.f * (gc1 * -U.mo[0] + 2.f * gc2 * -U.mo[1]);
        float gdl[6][2];
#pragma unroll
        for (int kk = 0; kk < 6; ++kk) {
            const float dx = U.dl[kk][0] - U.mo[0], dy = U.dl[kk][1] - U.mo[1];
            gdl[kk][0] = (2.f * gc0 * dx + gc1 * dy) * (1.f / 6.f);
            gdl[kk][1] = (gc1 * dx + 2.f * gc2 * dy) * (1.f / 6.f);
            gmx -= gdl[kk][0];
            gmy -= gdl[kk][1];
        }
        float sgx = 0.f, sgy = 0.f;  // total gradient on the six offsets (moves p_0 the other way)
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            float gD[3] = {0.f, 0.f, 0.f};
#pragma unroll
            for (int e = 0; e < 2; ++e) {
                const float sg = e == 0 ? 1.f : -1.f;
                const float gx = gdl[2 * a + e][0] + gmx * (1.f / 6.f);
                const float gy = gdl[2 * a + e][1] + gmy * (1.f / 6.f);
                sgx += gx;
                sgy += gy;
                const float xk = x0 + sg * U.D[a][0], yk = y0 + sg * U.D[a][1], zk = z0 + sg * U.D[a][2];
                float Jk[6];
                cam_jacobian(k, xk, yk, zk, Jk);
                const float g0 = gx * Jk[0] + gy * Jk[3], g1 = gx * Jk[1] + gy * Jk[4], g2 = gx * Jk[2] + gy * Jk[5];
                gmc[0] += g0;
                gmc[1] += g1;
                gmc[2] += g2;
                gD[0] += sg * g0;
                gD[1] += sg * g1;
                gD[2] += sg * g2;
            }
            // D_a = sqrt(3) s_a W R e_a
            const float h = kSqrt3 * P.s[a];
            A.s[a] += kSqrt3 * (U.WR[a] * gD[0] + U.WR[3 + a] * gD[1] + U.WR[6 + a] * gD[2]);
            for (int kk = 0; kk < 3; ++kk)
                gR[3 * kk + a] += h * (k.W[kk] * gD[0] + k.W[3 + kk] * gD[1] + k.W[6 + kk] * gD[2]);
        }
        // p_0 = proj(m_c) enters every offset with a minus sign
        float J0[6];
        cam_jacobian(k, x0, y0, z0, J0);
        gmc[0] -= sgx * J0[0] + sgy * J0[3];
        gmc[1] -= sgx * J0[1] + sgy * J0[4];
        gmc[2] -= sgx * J0[2] + sgy * J0[5];
    }
    for (int j = 0; j < 3; ++j) A.mu[j] += k.W[j] * gmc[0] + k.W[3 + j] * gmc[1] + k.W[6 + j] * gmc[2];
    rotation_adjoint(U.qn, gR, A.qn);
}

template <int DEG>
__global__ void __launch_bounds__(kBwdWarps * 32, 4) ut_project_bwd_kernel(
    const float *__restrict__ mu, const float *__restrict__ scale, const float *__restrict__ quat,
    const float *__restrict__ opac, const float *__restrict__ sh, int64_t n, CamSet cs, XprConfig cfg,
    const float *__restrict__ d_sd, float *__restrict__ gmu, float *__restrict__ gscale,
    float *__restrict__ gquat, float *__restrict__ gopac, float *__restrict__ gsh) {
    grid_dep_wait();
    constexpr int KC = (DEG + 1) * (DEG + 1) * 3;
    constexpr int LD = sh_ld<DEG>();
    extern __shared__ float s_utb[];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t base = ((int64_t)blockIdx.x * kBwdWarps + w) * 32;
    if (base >= n) return;
    const int nv = (int)min((int64_t)32, n - base);
    float *ssh = s_utb + (size_t)w * 2 * 32 * LD;
    float *sdsh = ssh + 32 * LD;
    stage_sh<DEG>(sh, base, nv, ssh);
    for (int c = 0; c < KC; ++c) sdsh[lane * LD + c] = 0.f;
    __syncwarp();
    const int64_t i = base + lane;
    if (i < n) {
        const Params P = load_params(mu, scale, quat, opac, i);
        Acc<DEG> A = {};
        float qinv = 0.f, qn[4] = {0.f, 0.f, 0.f, 0.f};
        for (int v = 0; v < cs.n_views; ++v) {
            const Cam k = make_cam(cs.cam[v], cfg);
            UtGeo U;
            ut_geometry(P, k, cfg.cov_dilation, U);
            if (!ut_footprint(U, P.o, k, cfg).vis) continue;
            const float4 *D4 = reinterpret_cast<const float4 *>(d_sd + ((size_t)v * n + i) * XPR_SD_FLOATS);
            ut_adjoint_view<DEG>(P, ssh + lane * LD, sdsh + lane * LD, U, k, cfg.cov_dilation, D4, A);
            qinv = U.qinv;
            for (int j = 0; j < 4; ++j) qn[j] = U.qn[j];
        }
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

// ---- ray-evaluated compositing ---------------------------------------------------------------
constexpr unsigned kFullUt = 0xffffffffu;
constexpr int kUtBatch = 256;     // list entries staged per shared-memory batch (forward)
constexpr int kUtBwdBatch = 128;  // the adjoint also keeps 16 accumulators per entry: half the batch
// Pixels per thread: (x, y + q h/PX), q = 0..PX-1, PX = min(4, tile pixels / 32), so that a
// tile's block is whole warps.
template <int TW, int TH>
__host__ __device__ constexpr int ut_px() {
    return (TW * TH) / 32 >= 4 ? 4 : (TW * TH) / 32;
}

struct UtConsts {
    int W, H, Wt, T;  // image size, tiles per row, tiles per view
    uint32_t n;       // records per launch: list entries >= n are ignored
    int batch;
    float at, amax, teps, bg0, bg1, bg2;
    int model;                 // camera: 0 pinhole, 1 fisheye
    float fx, fy, cx, cy, k[4];
};

// The coordinates a pixel is evaluated at: its centre (x + 0.5, y + 0.5) for the pinhole; for the
// fisheye the normalised image coordinates (d_x / d_z, d_y / d_z) of its ray d, whose angle theta from
// the axis solves theta_d(theta) = |m|, m = ((x + 0.5 - cx) / fx, (y + 0.5 - cy) / fy) (Newton's
// method).  Returns false for a ray at 1.5 rad or more from the axis (no finite coordinates).
template <bool FISH>
__device__ __forceinline__ bool ut_pixel_coord(const UtConsts &k, int x, int y, float &u, float &v) {
    const float X = (float)x + 0.5f, Y = (float)y + 0.5f;
    if (!FISH) {
        u = X;
        v = Y;
        return true;
    }
    const float mx = (X - k.cx) / k.fx, my = (Y - k.cy) / k.fy;
    const float td = sqrtf(mx * mx + my * my);
    if (td == 0.f) {
        u = v = 0.f;
        return true;
    }
    float th = td;
#pragma unroll 1
    for (int it = 0; it < 10; ++it) th -= (fish_thetad(k.k, th) - td) / fish_thetad_prime(k.k, th);
    if (!(th < 1.5f && th > 0.f)) return false;
    const float sc = tanf(th) / td;
    u = mx * sc;
    v = my * sc;
    return true;
}

// Staged entry: [p0x p0y A0x A0y] [A0z A1x A1y A1z] [o_c o'] [r g b |o_c|^2]
struct UtStage {
    float4 *u0, *u1, *u2, *u3;
    uint32_t *id;
};

__device__ __forceinline__ void ut_stage(const float *__restrict__ sd, const uint32_t *__restrict__ vals, int e,
                                         uint32_t n, const UtStage &S, int slot) {
    const uint32_t id = __ldg(vals + e);
    if (id < n) {
        const float4 *p = reinterpret_cast<const float4 *>(sd + (size_t)id * XPR_SD_FLOATS);
        S.u0[slot] = __ldg(p);
        S.u1[slot] = __ldg(p + 1);
        S.u2[slot] = __ldg(p + 2);
        S.u3[slot] = __ldg(p + 3);
    } else {  // never blended: o' = 0
        const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
        S.u0[slot] = z;
        S.u1[slot] = z;
        S.u2[slot] = z;
        S.u3[slot] = make_float4(0.f, 0.f, 0.f, 1.f);
    }
    if (S.id) S.id[slot] = id;
}

// Canonical offset a and the line minimum Q of one entry at pixel centre (cx, cy); the forward
// and the adjoint evaluate it with the same operations, so their alphas agree bit for bit.
struct UtEval {
    float dx, dy, a0, a1, a2, kap, Q;
};

__device__ __forceinline__ UtEval ut_eval(float cx, float cy, const float4 &u0, const float4 &u1, const float4 &u2,
                                          float rr) {
    UtEval r;
    r.dx = __fsub_rn(cx, u0.x);
    r.dy = __fsub_rn(cy, u0.y);
    r.a0 = __fmaf_rn(r.dx, u0.z, __fmul_rn(r.dy, u1.y));
    r.a1 = __fmaf_rn(r.dx, u0.w, __fmul_rn(r.dy, u1.z));
    r.a2 = __fmaf_rn(r.dx, u1.x, __fmul_rn(r.dy, u1.w));
    const float aa = __fmaf_rn(r.a2, r.a2, __fmaf_rn(r.a1, r.a1, __fmul_rn(r.a0, r.a0)));
    const float ar = __fmaf_rn(r.a2, u2.z, __fmaf_rn(r.a1, u2.y, __fmul_rn(r.a0, u2.x)));
    const float ab = __fsub_rn(aa, ar);
    const float bb = __fadd_rn(__fmaf_rn(-2.f, ar, aa), rr);
    r.kap = __fdividef(ab, bb);
    r.Q = __fmaf_rn(-r.kap, ab, aa);
    return r;
}

struct UtPixFwd {
    float cx, cy, T, r, g, b;
    int last;
    bool done;
};

struct UtWork {  // persistent scheduling: tiles list[0 .. count) taken through *counter
    const int *list;
    int *counter;
    int count;
};

template <int TW, int TH, bool FISH>
__device__ __forceinline__ void ut_fwd_tile(int gt, const float *__restrict__ sd, const uint32_t *__restrict__ vals,
                                            const int2 *__restrict__ ranges, const UtConsts &k,
                                            float *__restrict__ image, float *__restrict__ tfin,
                                            int *__restrict__ ncon, const UtStage &S) {
    constexpr int kUtPx = ut_px<TW, TH>();
    constexpr int NT = TW * TH / kUtPx, RS = TH / kUtPx;
    static_assert(NT % 32 == 0, "a tile's block must be whole warps");
    const float4 *s_u0 = S.u0, *s_u1 = S.u1, *s_u2 = S.u2, *s_u3 = S.u3;
    const int v = gt / k.T, tile = gt - v * k.T;
    const int tx = tile % k.Wt, ty = tile / k.Wt;
    const int t = threadIdx.x;
    const int px = tx * TW + t % TW, py = ty * TH + t / TW;
    const int2 rg = ranges[gt];
    const float col_x = (float)px + 0.5f;  // the pinhole's x coordinate, shared by the thread's pixels
    UtPixFwd P[kUtPx];
    bool in[kUtPx];
    bool all_done = true;
#pragma unroll
    for (int q = 0; q < kUtPx; ++q) {
        in[q] = px < k.W && py + q * RS < k.H;
        P[q] = UtPixFwd{0.f, 0.f, 1.f, 0.f, 0.f, 0.f, 0, !in[q]};
        if (in[q] && !ut_pixel_coord<FISH>(k, px, py + q * RS, P[q].cx, P[q].cy)) P[q].done = true;
        all_done &= P[q].done;
    }
    for (int base = rg.x; base < rg.y; base += k.batch) {
        if (__syncthreads_and(all_done)) break;
        const int cnt = min(k.batch, rg.y - base);
        for (int e = t; e < cnt; e += NT) ut_stage(sd, vals, base + e, k.n, S, e);
        __syncthreads();
        if (!all_done) {
            for (int j = 0; j < cnt; ++j) {
                const float4 u0 = s_u0[j], u1 = s_u1[j], u2 = s_u2[j], u3 = s_u3[j];
                const int pos = base + j - rg.x;
                all_done = true;
#pragma unroll
                for (int q = 0; q < kUtPx; ++q) {
                    UtPixFwd &p = P[q];
                    if (!p.done) {
                        const UtEval ev = ut_eval(FISH ? p.cx : col_x, p.cy, u0, u1, u2, u3.w);
                        const float G = ex2_approx(__fmul_rn(-0.5f * kLog2e, ev.Q));
                        if (G > kUtValid) {
                            const float og = __fmul_rn(u2.w, G);
                            const float al = fminf(k.amax, og);
                            if (al >= k.at) {
                                const float tt = __fmul_rn(p.T, __fsub_rn(1.f, al));
                                if (tt < k.teps) {
                                    p.done = true;
                                } else {
                                    const float w = al * p.T;
                                    p.r = fmaf(u3.x, w, p.r);
                                    p.g = fmaf(u3.y, w, p.g);
                                    p.b = fmaf(u3.z, w, p.b);
                                    p.T = tt;
                                    p.last = pos + 1;
                                }
                            }
                        }
                    }
                    all_done &= p.done;
                }
                if (all_done) break;
            }
        }
    }
    const int64_t HW = (int64_t)k.W * k.H;
    float *img = image + (int64_t)v * 3 * HW;
#pragma unroll
    for (int q = 0; q < kUtPx; ++q) {
        if (!in[q]) continue;
        const int64_t pix = (int64_t)(py + q * RS) * k.W + px;
        img[pix] = fmaf(P[q].T, k.bg0, P[q].r);
        img[HW + pix] = fmaf(P[q].T, k.bg1, P[q].g);
        img[2 * HW + pix] = fmaf(P[q].T, k.bg2, P[q].b);
        tfin[v * HW + pix] = P[q].T;
        ncon[v * HW + pix] = P[q].last;
    }
}

template <int TW, int TH, bool FISH>
__global__ void __launch_bounds__(TW *TH / ut_px<TW, TH>()) ut_render_fwd_kernel(
    const float *__restrict__ sd, const uint32_t *__restrict__ vals, const int2 *__restrict__ ranges, UtConsts k,
    float *__restrict__ image, float *__restrict__ tfin, int *__restrict__ ncon, UtWork w) {
    grid_dep_wait();
    __shared__ float4 s_u0[kUtBatch], s_u1[kUtBatch], s_u2[kUtBatch], s_u3[kUtBatch];
    const UtStage S = {s_u0, s_u1, s_u2, s_u3, nullptr};
    if (w.list == nullptr) {
        ut_fwd_tile<TW, TH, FISH>(blockIdx.x, sd, vals, ranges, k, image, tfin, ncon, S);
        return;
    }
    __shared__ int s_item;
    for (;;) {
        __syncthreads();  // the previous tile's last reads of shared memory are done
        if (threadIdx.x == 0) s_item = atomicAdd(w.counter, 1);
        __syncthreads();
        const int item = s_item;
        if (item >= w.count) break;
        ut_fwd_tile<TW, TH, FISH>(w.list[item], sd, vals, ranges, k, image, tfin, ncon, S);
    }
}

// Sum 16 per-lane values over the warp with 16 shuffles instead of 80: at each of the first four
// steps a lane keeps the half of its values selected by one bit of its lane index and sends the
// other half to its partner (xor 16, 8, 4, 2); a last xor 1 completes the sum.  Returns value
// (lane >> 1), held by lanes 2i and 2i + 1.
__device__ __forceinline__ float reduce_scatter16(const float *v, int lane) {
    const bool u16 = lane & 16, u8 = lane & 8, u4 = lane & 4, u2 = lane & 2;
    float b[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        const float send = u16 ? v[q] : v[q + 8];
        const float keep = u16 ? v[q + 8] : v[q];
        b[q] = keep + __shfl_xor_sync(kFullUt, send, 16);
    }
    float c[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const float send = u8 ? b[q] : b[q + 4];
        const float keep = u8 ? b[q + 4] : b[q];
        c[q] = keep + __shfl_xor_sync(kFullUt, send, 8);
    }
    float d[2];
#pragma unroll
    for (int q = 0; q < 2; ++q) {
        const float send = u4 ? c[q] : c[q + 2];
        const float keep = u4 ? c[q + 2] : c[q];
        d[q] = keep + __shfl_xor_sync(kFullUt, send, 4);
    }
    float e = (u2 ? d[1] : d[0]) + __shfl_xor_sync(kFullUt, u2 ? d[0] : d[1], 2);
    e += __shfl_xor_sync(kFullUt, e, 1);
    return e;
}

struct UtPixBwd {
    float cx, cy, T, g0, g1, g2, B;  // B = g . (colour behind the current entry)
    int last;
};

// Adds pixel P's partials for the entry at list position pos (back to front) into v[16]:
//   v[0..2] dL/da, v[3..5] dL/da dx, v[6..8] dL/da dy, v[9..11] dL/do_c, v[12] dL/do', v[13..15] dL/drgb.
__device__ __forceinline__ bool ut_adjoint(UtPixBwd &P, float cx, const float4 &u0, const float4 &u1,
                                           const float4 &u2, const float4 &u3, int pos, const UtConsts &k,
                                           float *v) {
    if (pos >= P.last) return false;
    const UtEval ev = ut_eval(cx, P.cy, u0, u1, u2, u3.w);
    const float G = ex2_approx(__fmul_rn(-0.5f * kLog2e, ev.Q));
    if (!(G > kUtValid)) return false;
    const float og = __fmul_rn(u2.w, G);
    const float al = fminf(k.amax, og);
    if (al < k.at) return false;
    const float inv = rcp_approx(1.f - al);
    const float Ti = P.T * inv;
    const float w = al * Ti;
    v[13] = fmaf(P.g0, w, v[13]);
    v[14] = fmaf(P.g1, w, v[14]);
    v[15] = fmaf(P.g2, w, v[15]);
    const float gc = fmaf(P.g0, u3.x, fmaf(P.g1, u3.y, P.g2 * u3.z));
    const float dal = fmaf(gc, Ti, -P.B * inv);
    P.B = fmaf(gc, w, P.B);
    P.T = Ti;
    if (og < k.amax) {
        v[12] = fmaf(dal, G, v[12]);
        const float dQ = -0.5f * dal * al;
        const float om = 1.f - ev.kap;
        const float e0 = om * ev.a0 + ev.kap * u2.x, e1 = om * ev.a1 + ev.kap * u2.y, e2 = om * ev.a2 + ev.kap * u2.z;
        const float fa = 2.f * om * dQ, fr = 2.f * ev.kap * dQ;
        const float g0 = fa * e0, g1 = fa * e1, g2 = fa * e2;
        v[0] += g0;
        v[1] += g1;
        v[2] += g2;
        v[3] = fmaf(g0, ev.dx, v[3]);
        v[4] = fmaf(g1, ev.dx, v[4]);
        v[5] = fmaf(g2, ev.dx, v[5]);
        v[6] = fmaf(g0, ev.dy, v[6]);
        v[7] = fmaf(g1, ev.dy, v[7]);
        v[8] = fmaf(g2, ev.dy, v[8]);
        v[9] = fmaf(fr, e0, v[9]);
        v[10] = fmaf(fr, e1, v[10]);
        v[11] = fmaf(fr, e2, v[11]);
    }
    return true;
}

template <int TW, int TH, bool FISH>
__device__ __forceinline__ void ut_bwd_tile(int gt, const float *__restrict__ sd, const uint32_t *__restrict__ vals,
                                            const int2 *__restrict__ ranges, const UtConsts &k,
                                            const float *__restrict__ tfin, const int *__restrict__ ncon,
                                            const float *__restrict__ dimg, float *__restrict__ d_sd,
                                            const UtStage &S, float (*s_acc)[kUtBwdBatch + 1], int *s_wmax) {
    constexpr int kUtPx = ut_px<TW, TH>();
    constexpr int NT = TW * TH / kUtPx, NW = NT / 32, RS = TH / kUtPx;
    static_assert(NT % 32 == 0, "a tile's block must be whole warps");
    const float4 *s_u0 = S.u0, *s_u1 = S.u1, *s_u2 = S.u2, *s_u3 = S.u3;
    const uint32_t *s_id = S.id;
    const int v = gt / k.T, tile = gt - v * k.T;
    const int tx = tile % k.Wt, ty = tile / k.Wt;
    const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
    const int px = tx * TW + t % TW, py = ty * TH + t / TW;
    const int2 rg = ranges[gt];
    const float col_x = (float)px + 0.5f;  // the pinhole's x coordinate, shared by the thread's pixels
    const int64_t HW = (int64_t)k.W * k.H;
    const float *tf = tfin + v * HW;
    const int *nc = ncon + v * HW;
    const float *di = dimg + (int64_t)v * 3 * HW;
    UtPixBwd P[kUtPx];
    int mylast = 0;
#pragma unroll
    for (int q = 0; q < kUtPx; ++q) {
        const int y = py + q * RS;
        const bool in = px < k.W && y < k.H;
        const int64_t pix = (int64_t)y * k.W + px;
        P[q] = UtPixBwd{0.f, 0.f, 1.f, 0.f, 0.f, 0.f, 0.f, 0};
        if (in && ut_pixel_coord<FISH>(k, px, y, P[q].cx, P[q].cy)) {
            P[q].T = tf[pix];
            P[q].last = nc[pix];
            P[q].g0 = di[pix];
            P[q].g1 = di[HW + pix];
            P[q].g2 = di[2 * HW + pix];
        }
        P[q].B = P[q].T * fmaf(P[q].g0, k.bg0, fmaf(P[q].g1, k.bg1, P[q].g2 * k.bg2));
        mylast = max(mylast, P[q].last);
    }
    const int wlast = __reduce_max_sync(kFullUt, mylast);
    if (lane == 0) s_wmax[wid] = wlast;
    __syncthreads();
    int bmax = 0;
#pragma unroll
    for (int w = 0; w < NW; ++w) bmax = max(bmax, s_wmax[w]);

    const int batch = min(k.batch, kUtBwdBatch);
    for (int end = rg.x + bmax; end > rg.x; end -= batch) {
        const int start = max(rg.x, end - batch);
        const int cnt = end - start;
        __syncthreads();
        for (int e = t; e < cnt; e += NT) {
            ut_stage(sd, vals, start + e, k.n, S, e);
#pragma unroll
            for (int c = 0; c < 16; ++c) s_acc[c][e] = 0.f;
        }
        __syncthreads();
        for (int j = cnt - 1; j >= 0; --j) {
            const int pos = start + j - rg.x;
            if (pos >= wlast) continue;  // warp-uniform: no pixel of this warp reached the entry
            float vv[16];
#pragma unroll
            for (int c = 0; c < 16; ++c) vv[c] = 0.f;
            const float4 u0 = s_u0[j], u1 = s_u1[j], u2 = s_u2[j], u3 = s_u3[j];
            bool hit = false;
#pragma unroll
            for (int q = 0; q < kUtPx; ++q) hit |= ut_adjoint(P[q], FISH ? P[q].cx : col_x, u0, u1, u2, u3, pos, k, vv);
            if (__any_sync(kFullUt, hit)) {
                const float r = reduce_scatter16(vv, lane);
                if ((lane & 1) == 0) atomicAdd(&s_acc[lane >> 1][j], r);
            }
        }
        __syncthreads();
        for (int e = t; e < cnt; e += NT) {
            float a[16];
            bool any = false;
#pragma unroll
            for (int c = 0; c < 16; ++c) {
                a[c] = s_acc[c][e];
                any |= (a[c] != 0.f);
            }
            if (any && s_id[e] < k.n) {
                const float4 u0 = s_u0[e], u1 = s_u1[e];
                // dp_0 = -(sum dL/da) . (A_0, A_1)
                const float dp0x = -(a[0] * u0.z + a[1] * u0.w + a[2] * u1.x);
                const float dp0y = -(a[0] * u1.y + a[1] * u1.z + a[2] * u1.w);
                float4 *d = reinterpret_cast<float4 *>(d_sd + (size_t)s_id[e] * XPR_SD_FLOATS);
                atomicAdd(d, make_float4(dp0x, dp0y, a[3], a[4]));
                atomicAdd(d + 1, make_float4(a[5], a[6], a[7], a[8]));
                atomicAdd(d + 2, make_float4(a[9], a[10], a[11], a[12]));
                atomicAdd(d + 3, make_float4(a[13], a[14], a[15], 0.f));
            }
        }
    }
}

template <int TW, int TH, bool FISH>
__global__ void __launch_bounds__(TW *TH / ut_px<TW, TH>()) ut_render_bwd_kernel(
    const float *__restrict__ sd, const uint32_t *__restrict__ vals, const int2 *__restrict__ ranges, UtConsts k,
    const float *__restrict__ tfin, const int *__restrict__ ncon, const float *__restrict__ dimg,
    float *__restrict__ d_sd, UtWork w) {
    grid_dep_wait();
    constexpr int NW = TW * TH / ut_px<TW, TH>() / 32;
    __shared__ float4 s_u0[kUtBwdBatch], s_u1[kUtBwdBatch], s_u2[kUtBwdBatch], s_u3[kUtBwdBatch];
    __shared__ uint32_t s_id[kUtBwdBatch];
    // rows padded by one float: the 16 lanes adding one entry's values hit 16 different banks
    __shared__ float s_acc[16][kUtBwdBatch + 1];
    __shared__ int s_wmax[NW];
    const UtStage S = {s_u0, s_u1, s_u2, s_u3, s_id};
    if (w.list == nullptr) {
        ut_bwd_tile<TW, TH, FISH>(blockIdx.x, sd, vals, ranges, k, tfin, ncon, dimg, d_sd, S, s_acc, s_wmax);
        return;
    }
    __shared__ int s_item;
    for (;;) {
        __syncthreads();  // the previous tile's last reads of shared memory are done
        if (threadIdx.x == 0) s_item = atomicAdd(w.counter, 1);
        __syncthreads();
        const int item = s_item;
        if (item >= w.count) break;
        ut_bwd_tile<TW, TH, FISH>(w.list[item], sd, vals, ranges, k, tfin, ncon, dimg, d_sd, S, s_acc, s_wmax);
    }
}

UtConsts make_ut_consts(const XprCamera &cam, const XprConfig &cfg, int64_t n) {
    UtConsts k;
    k.n = (uint32_t)n;
    k.W = cam.width;
    k.H = cam.height;
    k.Wt = tiles_x(cam, cfg);
    k.T = tiles_x(cam, cfg) * tiles_y(cam, cfg);
    k.batch = cfg.batch_depth > 0 ? min(cfg.batch_depth, kUtBatch) : kUtBatch;
    k.at = cfg.alpha_thresh;
    k.amax = cfg.alpha_max;
    k.teps = cfg.t_eps;
    k.bg0 = cfg.bg[0];
    k.bg1 = cfg.bg[1];
    k.bg2 = cfg.bg[2];
    k.model = cam.model;
    k.fx = cam.fx;
    k.fy = cam.fy;
    k.cx = cam.cx;
    k.cy = cam.cy;
    for (int i = 0; i < 4; ++i) k.k[i] = cam.dist[i];
    return k;
}

#define XPR_UT_TILE_DISPATCH(TWV, THV, ...)                                                       \
    if (cfg.tile_w == 16 && cfg.tile_h == 16) { constexpr int TWV = 16, THV = 16; __VA_ARGS__; }  \
    else if (cfg.tile_w == 8 && cfg.tile_h == 8) { constexpr int TWV = 8, THV = 8; __VA_ARGS__; } \
    else if (cfg.tile_w == 16 && cfg.tile_h == 8) { constexpr int TWV = 16, THV = 8; __VA_ARGS__; } \
    else { constexpr int TWV = 8, THV = 16; __VA_ARGS__; }

}  // namespace

int launch_ut_project_fwd_views(const XprPrims &p, int64_t n, const XprCamera *cams, int n_views,
                                const XprConfig &cfg, float *rec, float *sd, int32_t *bbox, int32_t *tc,
                                int32_t *isect_count, cudaStream_t st) {
    if (n == 0 || n_views == 0) return XPR_OK;
    const int tpb = kProjWarps * 32;
    const unsigned blocks = (unsigned)((n + tpb - 1) / tpb);
    const CamSet cs = make_camset(cams, n_views);
    XPR_DEG_DISPATCH(DEG, XPR_CUDA_TRY(launch_dependent(ut_project_fwd_kernel<DEG>, dim3(blocks), dim3(tpb),
                                                        (size_t)kProjWarps * 32 * sh_ld<DEG>() * sizeof(float), st,
                                                        p.mu, p.scale, p.quat, p.opacity, p.sh, n, cs, cfg, rec, sd,
                                                        reinterpret_cast<int4 *>(bbox), tc, isect_count)));
    XPR_LAUNCH_CHECK("ut_project_fwd_kernel");
    return XPR_OK;
}

int launch_ut_project_bwd_views(const XprPrims &p, int64_t n, const XprCamera *cams, int n_views,
                                const XprConfig &cfg, const float *d_sd, const XprPrimsGrad &g, cudaStream_t st) {
    if (n == 0 || n_views == 0) return XPR_OK;
    const int tpb = kBwdWarps * 32;
    const unsigned blocks = (unsigned)((n + tpb - 1) / tpb);
    const CamSet cs = make_camset(cams, n_views);
    cudaError_t attr = cudaSuccess;
    // the shared-memory size is a constant of each instantiation, so every caller sets the same limit
    XPR_DEG_DISPATCH(DEG, {
        const size_t smem = (size_t)kBwdWarps * 2 * 32 * sh_ld<DEG>() * sizeof(float);
        attr = cudaFuncSetAttribute(ut_project_bwd_kernel<DEG>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)smem);
        if (attr == cudaSuccess)
            XPR_CUDA_TRY(launch_dependent(ut_project_bwd_kernel<DEG>, dim3(blocks), dim3(tpb), smem, st, p.mu, p.scale,
                                          p.quat, p.opacity, p.sh, n, cs, cfg, d_sd, g.mu, g.scale, g.quat, g.opacity,
                                          g.sh));
    });
    XPR_CUDA_TRY(attr);
    XPR_LAUNCH_CHECK("ut_project_bwd_kernel");
    return XPR_OK;
}

template <typename KernelT>
int ut_persistent_grid(KernelT kernel, int threads, int items) {
    int dev = 0, sms = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return items;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return items;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, 0) != cudaSuccess || per_sm < 1)
        per_sm = 1;
    return max(1, min(items, sms * per_sm));
}

// worklist/counter NULL: one block per tile over n_views * T tiles.  Otherwise a persistent grid
// walks worklist[0 .. n_views * T); *counter is zeroed here.
int launch_ut_render_fwd(const float *sd, int64_t n, const uint32_t *vals, const int32_t *ranges, int n_views,
                         const XprCamera &cam, const XprConfig &cfg, float *image, float *t_final,
                         int32_t *n_contrib, const int32_t *worklist, int32_t *counter, cudaStream_t st) {
    const UtConsts k = make_ut_consts(cam, cfg, n);
    const int items = n_views * k.T;
    if (items == 0) return XPR_OK;
    const int2 *rg = reinterpret_cast<const int2 *>(ranges);
    const UtWork w = {worklist, counter, items};
    if (worklist) XPR_CUDA_TRY(cudaMemsetAsync(counter, 0, sizeof(int32_t), st));
    // the camera model is a template argument: the pinhole kernels carry no unprojection code
    if (cam.model == 1) {
        XPR_UT_TILE_DISPATCH(TW, TH, {
            const int threads = TW * TH / ut_px<TW, TH>();
            const int grid = worklist ? ut_persistent_grid(ut_render_fwd_kernel<TW, TH, true>, threads, items) : items;
            XPR_CUDA_TRY(launch_dependent(ut_render_fwd_kernel<TW, TH, true>, dim3(grid), dim3(threads), 0, st, sd,
                                          vals, rg, k, image, t_final, n_contrib, w));
        });
    } else {
        XPR_UT_TILE_DISPATCH(TW, TH, {
            const int threads = TW * TH / ut_px<TW, TH>();
            const int grid = worklist ? ut_persistent_grid(ut_render_fwd_kernel<TW, TH, false>, threads, items) : items;
            XPR_CUDA_TRY(launch_dependent(ut_render_fwd_kernel<TW, TH, false>, dim3(grid), dim3(threads), 0, st, sd,
                                          vals, rg, k, image, t_final, n_contrib, w));
        });
    }
    XPR_LAUNCH_CHECK("ut_render_fwd_kernel");
    return XPR_OK;
}

int launch_ut_render_bwd(const float *sd, int64_t n, const uint32_t *vals, const int32_t *ranges, int n_views,
                         const XprCamera &cam, const XprConfig &cfg, const float *t_final, const int32_t *n_contrib,
                         const float *d_image, float *d_sd, const int32_t *worklist, int32_t *counter,
                         cudaStream_t st) {
    XPR_CUDA_TRY(cudaMemsetAsync(d_sd, 0, (size_t)n * XPR_SD_FLOATS * sizeof(float), st));
    const UtConsts k = make_ut_consts(cam, cfg, n);
    const int items = n_views * k.T;
    if (items == 0) return XPR_OK;
    const int2 *rg = reinterpret_cast<const int2 *>(ranges);
    const UtWork w = {worklist, counter, items};
    if (worklist) XPR_CUDA_TRY(cudaMemsetAsync(counter, 0, sizeof(int32_t), st));
    if (cam.model == 1) {
        XPR_UT_TILE_DISPATCH(TW, TH, {
            const int threads = TW * TH / ut_px<TW, TH>();
            const int grid = worklist ? ut_persistent_grid(ut_render_bwd_kernel<TW, TH, true>, threads, items) : items;
            XPR_CUDA_TRY(launch_dependent(ut_render_bwd_kernel<TW, TH, true>, dim3(grid), dim3(threads), 0, st, sd,
                                          vals, rg, k, t_final, n_contrib, d_image, d_sd, w));
        });
    } else {
        XPR_UT_TILE_DISPATCH(TW, TH, {
            const int threads = TW * TH / ut_px<TW, TH>();
            const int grid = worklist ? ut_persistent_grid(ut_render_bwd_kernel<TW, TH, false>, threads, items) : items;
            XPR_CUDA_TRY(launch_dependent(ut_render_bwd_kernel<TW, TH, false>, dim3(grid), dim3(threads), 0, st, sd,
                                          vals, rg, k, t_final, n_contrib, d_image, d_sd, w));
        });
    }
    XPR_LAUNCH_CHECK("ut_render_bwd_kernel");
    return XPR_OK;
}

}  // namespace xpr
