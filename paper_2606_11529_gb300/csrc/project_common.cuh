// Helpers shared by the projection kernels of 3DGS (project.cu) and 3DGUT (ut.cu): spherical
// harmonics, the camera, the rotation of a quaternion and its adjoint, per-warp staging of SH
// coefficients, and the view-dependent colour with its adjoint.  Everything lives in an unnamed
// namespace, so each translation unit keeps its own inlined copy.
#pragma once

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
    int model;   // 0 pinhole, 1 fisheye
    float k[4];  // fisheye radial coefficients
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
    k.model = c.model;
    for (int i = 0; i < 4; ++i) k.k[i] = c.dist[i];
    return k;
}

// Camera point m_c = W mu + t with every operation rounded to float32 in a fixed order and no fused
// multiply-add: m_c,i = ((W_i0 x + W_i1 y) + W_i2 z) + t_i.  The depth sort key comes from it
// (camera z, or the Euclidean distance below), so the order of the tile lists is a reproducible
// integer decision: the same float32 operations give the same key bits on any IEEE machine.
__device__ __forceinline__ void cam_point(const Cam &k, const float *m, float *mc) {
#pragma unroll
    for (int i = 0; i < 3; ++i)
        mc[i] = __fadd_rn(__fadd_rn(__fadd_rn(__fmul_rn(k.W[3 * i], m[0]), __fmul_rn(k.W[3 * i + 1], m[1])),
                                    __fmul_rn(k.W[3 * i + 2], m[2])),
                          k.t[i]);
}

// Euclidean distance of a camera point, rounded as sqrt((x x + y y) + z z) with no fused operation.
__device__ __forceinline__ float euclid_depth(const float *mc) {
    return __fsqrt_rn(__fadd_rn(__fadd_rn(__fmul_rn(mc[0], mc[0]), __fmul_rn(mc[1], mc[1])), __fmul_rn(mc[2], mc[2])));
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

struct CamSet {
    XprCamera cam[kMaxViews];
    int n_views;
};

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
// A full warp whose rows start on a 16-byte boundary loads them as float4, every load of a lane
// issued before its first shared-memory store (12 loads in flight per lane at degree 3).
template <int DEG>
__device__ __forceinline__ void stage_sh(const float *__restrict__ sh, int64_t base, int nv, float *ssh) {
    constexpr int KC = (DEG + 1) * (DEG + 1) * 3;
    constexpr int LD = sh_ld<DEG>();
    constexpr int F4 = 8 * KC;          // float4 of a full warp's rows (32 KC floats)
    constexpr int PER = (F4 + 31) / 32;  // per lane
    const int lane = threadIdx.x & 31;
    const float *gs = sh + base * KC;
    if (nv == 32 && (reinterpret_cast<uintptr_t>(gs) & 15) == 0) {
        float4 r[PER];
#pragma unroll
        for (int it = 0; it < PER; ++it) {
            const int u = lane + 32 * it;
            if (u < F4) r[it] = __ldg(reinterpret_cast<const float4 *>(gs) + u);
        }
#pragma unroll
        for (int it = 0; it < PER; ++it) {
            const int u = lane + 32 * it;
            if (u < F4) {
                const float v4[4] = {r[it].x, r[it].y, r[it].z, r[it].w};
#pragma unroll
                for (int c4 = 0; c4 < 4; ++c4) {
                    const int e = 4 * u + c4;
                    const int pi = e / KC;
                    ssh[pi * LD + (e - pi * KC)] = v4[c4];
                }
            }
        }
    } else {
        for (int e = lane; e < nv * KC; e += 32) {
            const int pi = e / KC;
            ssh[pi * LD + (e - pi * KC)] = __ldg(gs + e);
        }
    }
    __syncwarp();
}

// Writes the staged rows of a warp's nv primitives (row stride LD in shared memory) to the
// contiguous rows at go, coalesced (float4 stores for a full warp on a 16-byte boundary).
template <int DEG>
__device__ __forceinline__ void write_sh_rows(const float *ssh, int nv, float *__restrict__ go) {
    constexpr int KC = (DEG + 1) * (DEG + 1) * 3;
    constexpr int LD = sh_ld<DEG>();
    constexpr int F4 = 8 * KC;
    constexpr int PER = (F4 + 31) / 32;
    const int lane = threadIdx.x & 31;
    if (nv == 32 && (reinterpret_cast<uintptr_t>(go) & 15) == 0) {
#pragma unroll
        for (int it = 0; it < PER; ++it) {
            const int u = lane + 32 * it;
            if (u < F4) {
                float v4[4];
#pragma unroll
                for (int c4 = 0; c4 < 4; ++c4) {
                    const int e = 4 * u + c4;
                    const int pi = e / KC;
                    v4[c4] = ssh[pi * LD + (e - pi * KC)];
                }
                reinterpret_cast<float4 *>(go)[u] = make_float4(v4[0], v4[1], v4[2], v4[3]);
            }
        }
    } else {
        for (int e = lane; e < nv * KC; e += 32) {
            const int pi = e / KC;
            go[e] = ssh[pi * LD + (e - pi * KC)];
        }
    }
}

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

// Accumulators of a projection adjoint over views.  The quaternion gradient is kept with respect to
// the normalised quaternion and projected through the normalisation once at the end.
template <int DEG>
struct Acc {
    float mu[3], s[3], qn[4], o;
};
constexpr int kBwdWarps = 4;  // warps per block of the projection adjoints

// Colour adjoint (the shared tail of both projection adjoints): dL/dsh_k = Y_k g where the colour
// was not clamped at 0, and dL/dmu through the direction d = (mu - c)/|mu - c|: the basis gradient
// projected on the tangent plane and divided by |mu - c|.
template <int DEG>
__device__ __forceinline__ void colour_adjoint(const Params &P, const float *shi, float *dsh, const Cam &k,
                                               const float *drgb, float *gmu) {
    constexpr int K = (DEG + 1) * (DEG + 1);
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
    gmu[0] += (gdir.x - ux * dd) * vinv;
    gmu[1] += (gdir.y - uy * dd) * vinv;
    gmu[2] += (gdir.z - uz * dd) * vinv;
}

// dL/dqn += partials of the unit-quaternion rotation matrix R(qn) (quat_to_rot) against gR.
__device__ __forceinline__ void rotation_adjoint(const float *qn, const float *gR, float *gqn) {
    const float w = qn[0], qx = qn[1], qy = qn[2], qz = qn[3];
    gqn[0] += 2.f * (-qz * gR[1] + qy * gR[2] + qz * gR[3] - qx * gR[5] - qy * gR[6] + qx * gR[7]);
    gqn[1] += 2.f * (qy * gR[1] + qz * gR[2] + qy * gR[3] - 2.f * qx * gR[4] - w * gR[5] + qz * gR[6] +
                     w * gR[7] - 2.f * qx * gR[8]);
    gqn[2] += 2.f * (-2.f * qy * gR[0] + qx * gR[1] + w * gR[2] + qx * gR[3] + qz * gR[5] - w * gR[6] +
                     qz * gR[7] - 2.f * qy * gR[8]);
    gqn[3] += 2.f * (-2.f * qz * gR[0] - w * gR[1] + qx * gR[2] + w * gR[3] - 2.f * qz * gR[4] + qy * gR[5] +
                     qx * gR[6] + qy * gR[7]);
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
}  // namespace xpr
