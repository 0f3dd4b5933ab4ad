// LinPrim (Appendix, implementation of XPR-LinPrim): octahedra {x : ||S^-1 R^T (x - mu)||_1 <= 1}
// with homogeneous density, projected as four slab pairs, evaluated by slab intersection along the
// pixel ray, culled per tile by the chord bound of Eq. (linprim_tile_cull); and the adjoints.
//
// Projection (per primitive and view):
//   m_c = W mu + t, d = |m_c|, mu_2D = (fx x/z + cx, fy y/z + cy);
//   A = J3 W R diag(s), J3 = [[fx/z, 0, -fx x/z^2], [0, fy/z, -fy y/z^2], m_c^T / d] (the pinhole
//   Jacobian plus the Euclidean-distance row, so tau is depth along the ray); c0, c1, c2 = rows of
//   A^-1; slab normals n_i = c0 + e1 c1 + e2 c2, (e1, e2) = (+,+), (+,-), (-,+), (-,-);
//   extents ex = max_k |A_0k|, ey = max_k |A_1k| (the six vertices), box of mu_2D - 0.5;
//   sigma = -log(1 - 0.99 clip(o, 0, 0.999)) / (2 min s); depth = d; visible iff z > z_near,
//   d > z_near, min s > 0, r > 0, tc > 0.
// Shader data sd[20] (also the cull's data, so the binning reads it instead of the record):
//   [mu_2D.x mu_2D.y sigma req] then per slab (p, q, h) = (n_x / n_z, n_y / n_z, 1 / |n_z|) (p = q = 0,
//   h = inf when |n_z| < 1e-10), then [r g b 0]; req = -log(1 - alpha_t).  With (dX, dY) the pixel
//   centre minus mu_2D, slab i bounds tau to m_i -+ h_i, m_i = -(p_i dX + q_i dY).
// Record rec[12]: mu_2D [0,1], rgb [6..8], depth d [9], visible [11] (the depth order reads it).
// Evaluate: dtau = min_i (m_i + h_i) - max_i (m_i - h_i); alpha = 1 - exp(-sigma dtau) if dtau > 0.
// Cull: keep the tile iff sigma max(0, min_{i,j} [h_i + h_j + max_corners (m_i - m_j)]) >= req over
// the tile's four pixel-centre corners, in FP32 with one correctly rounded operation per step.
#include "project_common.cuh"

namespace xpr {
namespace {

constexpr float kLpEps = 1e-10f;
// signs (e1, e2) of slab i: (+,+), (+,-), (-,+), (-,-)
__host__ __device__ constexpr float es1(int i) { return i < 2 ? 1.f : -1.f; }
__host__ __device__ constexpr float es2(int i) { return (i & 1) ? -1.f : 1.f; }

struct LpGeo {
    float qn[4], qinv, R[9];
    float mc[3], d;
    float J[9], M[9], A[9], Ai[9];
    float n[4][3], pqh[4][3];
    float ex, ey, smin, oc, sigma, mx, my;
    int kmin;
    bool oclip, front;
};

__device__ __forceinline__ void lp_geometry(const Params &P, const Cam &k, LpGeo &G) {
    const float qq = P.q[0] * P.q[0] + P.q[1] * P.q[1] + P.q[2] * P.q[2] + P.q[3] * P.q[3];
    G.qinv = rsqrtf(qq);
    for (int i = 0; i < 4; ++i) G.qn[i] = P.q[i] * G.qinv;
    quat_to_rot(G.qn[0], G.qn[1], G.qn[2], G.qn[3], G.R);
    cam_point(k, P.m, G.mc);
    const float x = G.mc[0], y = G.mc[1], z = G.mc[2];
    G.d = euclid_depth(G.mc);
    G.kmin = P.s[1] < P.s[0] ? 1 : 0;
    if (P.s[2] < P.s[G.kmin]) G.kmin = 2;
    G.smin = P.s[G.kmin];
    G.oc = fminf(fmaxf(P.o, 0.f), 0.999f);
    G.oclip = !(P.o > 0.f && P.o < 0.999f);
    G.sigma = -log1pf(-0.99f * G.oc) / (2.f * G.smin);
    G.front = (z > k.z_near) && (G.d > k.z_near) && (G.smin > 0.f);
    if (!G.front) return;
    const float iz = 1.f / z, id = 1.f / G.d;
    G.mx = k.fx * (x * iz) + k.cx;
    G.my = k.fy * (y * iz) + k.cy;
    const float J[9] = {k.fx * iz, 0.f, -k.fx * x * iz * iz, 0.f, k.fy * iz, -k.fy * y * iz * iz, x * id, y * id, z * id};
    for (int i = 0; i < 9; ++i) G.J[i] = J[i];
    for (int i = 0; i < 3; ++i)
        for (int c = 0; c < 3; ++c)
            G.M[3 * i + c] = k.W[3 * i] * G.R[c] + k.W[3 * i + 1] * G.R[3 + c] + k.W[3 * i + 2] * G.R[6 + c];
    for (int i = 0; i < 3; ++i)
        for (int c = 0; c < 3; ++c)
            G.A[3 * i + c] = (J[3 * i] * G.M[c] + J[3 * i + 1] * G.M[3 + c] + J[3 * i + 2] * G.M[6 + c]) * P.s[c];
    const float *A = G.A;
    const float c00 = A[4] * A[8] - A[5] * A[7], c01 = A[5] * A[6] - A[3] * A[8], c02 = A[3] * A[7] - A[4] * A[6];
    const float det = A[0] * c00 + A[1] * c01 + A[2] * c02;
    const float idet = 1.f / det;
    G.Ai[0] = c00 * idet;
    G.Ai[1] = (A[2] * A[7] - A[1] * A[8]) * idet;
    G.Ai[2] = (A[1] * A[5] - A[2] * A[4]) * idet;
    G.Ai[3] = c01 * idet;
    G.Ai[4] = (A[0] * A[8] - A[2] * A[6]) * idet;
    G.Ai[5] = (A[2] * A[3] - A[0] * A[5]) * idet;
    G.Ai[6] = c02 * idet;
    G.Ai[7] = (A[1] * A[6] - A[0] * A[7]) * idet;
    G.Ai[8] = (A[0] * A[4] - A[1] * A[3]) * idet;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        for (int c = 0; c < 3; ++c) G.n[i][c] = G.Ai[c] + es1(i) * G.Ai[3 + c] + es2(i) * G.Ai[6 + c];
        const bool ok = fabsf(G.n[i][2]) >= kLpEps;
        const float inz = ok ? 1.f / G.n[i][2] : 0.f;
        G.pqh[i][0] = G.n[i][0] * inz;
        G.pqh[i][1] = G.n[i][1] * inz;
        G.pqh[i][2] = ok ? fabsf(inz) : __int_as_float(0x7f800000);
    }
    G.ex = fmaxf(fabsf(A[0]), fmaxf(fabsf(A[1]), fabsf(A[2])));
    G.ey = fmaxf(fabsf(A[3]), fmaxf(fabsf(A[4]), fabsf(A[5])));
}

// The cull decision for the tile with pixel-centre corners (X0, Y0) .. (X1, Y1) from the stored
// shader data S[0..15]; every step one correctly rounded IEEE operation, no contraction.
__device__ __forceinline__ bool lp_keep(const float *S, float X0, float Y0, float X1, float Y1) {
    const float dX[2] = {__fsub_rn(X0, S[0]), __fsub_rn(X1, S[0])};
    const float dY[2] = {__fsub_rn(Y0, S[1]), __fsub_rn(Y1, S[1])};
    float m[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int c = 0; c < 4; ++c)
            m[i][c] = -__fadd_rn(__fmul_rn(S[4 + 3 * i], dX[c >> 1]), __fmul_rn(S[5 + 3 * i], dY[c & 1]));
    float best = __int_as_float(0x7f800000);
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            float g = __fsub_rn(m[i][0], m[j][0]);
#pragma unroll
            for (int c = 1; c < 4; ++c) g = fmaxf(g, __fsub_rn(m[i][c], m[j][c]));
            g = __fadd_rn(__fadd_rn(g, S[6 + 3 * i]), S[6 + 3 * j]);
            best = fminf(best, g);
        }
    best = fmaxf(best, 0.f);
    return __fmul_rn(S[2], best) >= S[3];
}

__device__ __forceinline__ void tile_corners(const Grid &g, int tx, int ty, float &X0, float &Y0, float &X1,
                                             float &Y1) {
    X0 = (float)(tx * g.tw) + 0.5f;
    Y0 = (float)(ty * g.th) + 0.5f;
    X1 = (float)min(tx * g.tw + g.tw - 1, g.W - 1) + 0.5f;
    Y1 = (float)min(ty * g.th + g.th - 1, g.H - 1) + 0.5f;
}

// The tiles of the warp's 32 boxes (one per lane: area tiles in row-major slots of box bb, cull data
// S) are walked 32 at a time, flattened over the lanes: lane l tests slot f0 + l of the flattened
// list with its owner's data (shuffled), so large boxes do not serialise a warp.  Returns the number
// of kept tiles of the lane's own box.  With EMIT it also writes them, in slot order, at
// cursor, cursor + 1, ... (never at or past end): a kept slot's position is its owner's cursor plus
// the kept slots before it in the owner's run of lanes.  Every lane of the warp must call this.
template <bool EMIT>
__device__ __forceinline__ int lp_walk(const float *S, int4 bb, int area, const Grid &g, int64_t cursor, int64_t end,
                                       uint32_t tbase, uint32_t depth_bits, uint32_t id, uint64_t *keys,
                                       uint32_t *tiles, uint32_t *vals) {
    const int lane = threadIdx.x & 31;
    const int incl = warp_incl_scan(area);
    const int total = __shfl_sync(kFullMask, incl, 31);
    const int excl = incl - area;
    const int bw = max(bb.z - bb.x, 1);
    int cnt = 0;
    for (int f0 = 0; f0 < total; f0 += 32) {
        const int f = f0 + lane;
        const int p = lane_of(incl, f);
        float T[16];
#pragma unroll
        for (int c = 0; c < 16; ++c) T[c] = __shfl_sync(kFullMask, S[c], p);
        const int pexcl = __shfl_sync(kFullMask, excl, p);
        const int pbx = __shfl_sync(kFullMask, bb.x, p), pby = __shfl_sync(kFullMask, bb.y, p);
        const int pbw = __shfl_sync(kFullMask, bw, p);
        bool keep = false;
        int tx = 0, ty = 0;
        if (f < total) {
            const int r = f - pexcl, q = r / pbw;
            ty = pby + q;
            tx = pbx + (r - q * pbw);
            float X0, Y0, X1, Y1;
            tile_corners(g, tx, ty, X0, Y0, X1, Y1);
            keep = lp_keep(T, X0, Y0, X1, Y1);
        }
        const unsigned bal = __ballot_sync(kFullMask, keep);
        if (EMIT) {
            const int64_t pcur = __shfl_sync(kFullMask, cursor, p);
            const int64_t pend = __shfl_sync(kFullMask, end, p);
            const uint32_t ptb = __shfl_sync(kFullMask, tbase, p), pdb = __shfl_sync(kFullMask, depth_bits, p);
            const uint32_t pid = __shfl_sync(kFullMask, id, p);
            const int plo = max(pexcl - f0, 0);  // first lane of the owner's run in this step
            const unsigned before = bal & ((1u << lane) - 1u) & ~((1u << plo) - 1u);
            const int64_t pos = pcur + __popc(before);
            if (keep && pos < pend) {
                const uint32_t t = ptb + (uint32_t)(ty * g.Wt + tx);
                if (keys) keys[pos] = ((uint64_t)t << 32) | pdb;
                if (tiles) tiles[pos] = t;
                vals[pos] = pid;
            }
        }
        // this lane's own run of slots in the step: lanes [lo, hi]
        const int lo = max(excl - f0, 0), hi = min(incl - 1 - f0, 31);
        if (area > 0 && lo <= 31 && hi >= 0 && lo <= hi) {
            const unsigned run = (hi == 31 ? 0xffffffffu : ((1u << (hi + 1)) - 1u)) & ~((1u << lo) - 1u);
            const int k = __popc(bal & run);
            cnt += k;
            cursor += k;
        }
    }
    return cnt;
}

template <int DEG>
__global__ void __launch_bounds__(kProjWarps * 32) lp_project_fwd_kernel(
    const float *__restrict__ mu, const float *__restrict__ scale, const float *__restrict__ quat,
    const float *__restrict__ opac, const float *__restrict__ sh, int64_t n, CamSet cs, XprConfig cfg,
    float *__restrict__ rec, float *__restrict__ sd, int4 *__restrict__ bbox, int *__restrict__ tcount,
    int *__restrict__ isect_count) {
    grid_dep_wait();
    constexpr int LD = sh_ld<DEG>();
    extern __shared__ float s_lpf[];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t base = ((int64_t)blockIdx.x * kProjWarps + w) * 32;
    if (base >= n) return;
    const int nv = (int)min((int64_t)32, n - base);
    float *ssh = s_lpf + (size_t)w * 32 * LD;
    stage_sh<DEG>(sh, base, nv, ssh);
    const int64_t i = base + lane;
    const bool valid = i < n;
    Params P = {};
    if (valid) P = load_params(mu, scale, quat, opac, i);
    const float req = -log1pf(-cfg.alpha_thresh);
    for (int v = 0; v < cs.n_views; ++v) {
        const Cam k = make_cam(cs.cam[v], cfg);
        const int64_t out = (int64_t)v * n + i;
        float S[16] = {};
        int4 bb = make_int4(0, 0, 0, 0);
        int tc = 0;
        if (valid) {
            LpGeo G;
            lp_geometry(P, k, G);
            float4 *o4 = reinterpret_cast<float4 *>(rec + (size_t)out * XPR_REC_FLOATS);
            float4 *s4 = reinterpret_cast<float4 *>(sd + (size_t)out * XPR_LP_SD_FLOATS);
            const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
            bool vis = false;
            if (G.front) {
                const float Wt = (float)((k.width + cfg.tile_w - 1) / cfg.tile_w);
                const float Ht = (float)((k.height + cfg.tile_h - 1) / cfg.tile_h);
                const float tw = (float)cfg.tile_w, th = (float)cfg.tile_h;
                const float bx = G.mx - 0.5f, by = G.my - 0.5f;  // ray offset: pixel centres at +0.5
                bb.x = (int)fminf(fmaxf(floorf((bx - G.ex) / tw), 0.f), Wt);
                bb.y = (int)fminf(fmaxf(floorf((by - G.ey) / th), 0.f), Ht);
                bb.z = (int)fminf(fmaxf(floorf((bx + G.ex) / tw) + 1.f, 0.f), Wt);
                bb.w = (int)fminf(fmaxf(floorf((by + G.ey) / th) + 1.f, 0.f), Ht);
                tc = (bb.z - bb.x) * (bb.w - bb.y);
                vis = (fmaxf(G.ex, G.ey) > 0.f) && (tc > 0);
            }
            if (!vis) {
                o4[0] = z4;
                o4[1] = z4;
                o4[2] = make_float4(0.f, G.d, 0.f, 0.f);
                for (int c = 0; c < 5; ++c) s4[c] = z4;
                bbox[out] = make_int4(0, 0, 0, 0);
                tcount[out] = 0;
                bb = make_int4(0, 0, 0, 0);
                tc = 0;
            } else {
                float col[3];
                sh_colour<DEG>(P, ssh + lane * LD, k, col);
                for (int c = 0; c < 3; ++c) col[c] = fmaxf(col[c], 0.f);
                S[0] = G.mx;
                S[1] = G.my;
                S[2] = G.sigma;
                S[3] = req;
                for (int q = 0; q < 4; ++q)
                    for (int c = 0; c < 3; ++c) S[4 + 3 * q + c] = G.pqh[q][c];
                o4[0] = make_float4(G.mx, G.my, 0.f, 0.f);
                o4[1] = make_float4(0.f, 0.f, col[0], col[1]);
                o4[2] = make_float4(col[2], G.d, 0.f, 1.f);
                for (int c = 0; c < 4; ++c) s4[c] = make_float4(S[4 * c], S[4 * c + 1], S[4 * c + 2], S[4 * c + 3]);
                s4[4] = make_float4(col[0], col[1], col[2], 0.f);
                bbox[out] = bb;
                tcount[out] = tc;
            }
        }
        if (isect_count) {  // kept tiles, with the binning's cull on the stored values
            const int cnt = lp_walk<false>(S, bb, tc, make_grid(cs.cam[v], cfg), 0, 0, 0, 0, 0, nullptr, nullptr,
                                           nullptr);
            if (valid) isect_count[out] = cnt;
        }
    }
}

__device__ __forceinline__ void lp_load16(const float *__restrict__ sd, int64_t i, float *S) {
    const float4 *p = reinterpret_cast<const float4 *>(sd + (size_t)i * XPR_LP_SD_FLOATS);
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        const float4 v = __ldg(p + c);
        S[4 * c] = v.x;
        S[4 * c + 1] = v.y;
        S[4 * c + 2] = v.z;
        S[4 * c + 3] = v.w;
    }
}

__device__ __forceinline__ int lp_box(const int4 *__restrict__ bbox, const int *__restrict__ tcount, int64_t i,
                                      const Grid &g, int4 &bb) {
    bb = make_int4(0, 0, 0, 0);
    if (tcount[i] <= 0) return 0;
    bb = bbox[i];
    bb.x = max(bb.x, 0);  // never leave the tile grid, whatever the caller's boxes say
    bb.y = max(bb.y, 0);
    bb.z = min(bb.z, g.Wt);
    bb.w = min(bb.w, g.Ht);
    return (bb.z > bb.x && bb.w > bb.y) ? 1 : 0;
}

// Binning count and emit passes over positions j (primitive order[j]).  Warp w of the grid takes the
// 32 positions w, w + nw, w + 2 nw, ... (nw warps in all), so every warp gets primitives from all
// depths (in depth order the near-camera boxes, which hold most pairs, are neighbours).
template <bool EMIT>
__global__ void __launch_bounds__(256) lp_bin_kernel(const float *__restrict__ rec, const float *__restrict__ sd,
                                                     const int4 *__restrict__ bbox, const int *__restrict__ tcount,
                                                     const int *__restrict__ order, int64_t n, Grid g,
                                                     int32_t *__restrict__ counts, const int32_t *__restrict__ offsets,
                                                     uint64_t *__restrict__ keys, uint32_t *__restrict__ tiles,
                                                     uint32_t *__restrict__ vals, int64_t per_view) {
    grid_dep_wait();
    const int lane = threadIdx.x & 31;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t j = w + (int64_t)lane * nw;
    const bool valid = j < n;
    const int64_t i = valid ? (order ? order[j] : j) : 0;
    int4 bb = make_int4(0, 0, 0, 0);
    int area = 0;
    float S[16] = {};
    if (valid && lp_box(bbox, tcount, i, g, bb)) {
        area = (bb.z - bb.x) * (bb.w - bb.y);
        lp_load16(sd, i, S);
    }
    if (!EMIT) {
        const int cnt = lp_walk<false>(S, bb, area, g, 0, 0, 0, 0, 0, nullptr, nullptr, nullptr);
        if (valid) counts[j] = cnt;
        return;
    }
    const int64_t cur = valid ? offsets[j] : 0, end = valid ? offsets[j + 1] : 0;
    const uint32_t depth_bits = area > 0 ? __float_as_uint(__ldg(rec + (size_t)i * XPR_REC_FLOATS + 9)) : 0u;
    const uint32_t tbase = per_view > 0 ? (uint32_t)(i / per_view) * (uint32_t)(g.Wt * g.Ht) : 0u;
    lp_walk<true>(S, bb, area, g, cur, end, tbase, depth_bits, (uint32_t)i, keys, tiles, vals);
}

// ---- compositing -----------------------------------------------------------------------------
constexpr unsigned kFullLp = 0xffffffffu;
constexpr int kLpBatch = 128;     // entries staged per batch (forward; 128 rather than 256: 78 instead of 94 registers, 10% faster)
constexpr int kLpBwdBatch = 128;  // the adjoint also keeps 20 accumulators per entry
template <int TW, int TH>
__host__ __device__ constexpr int lp_px() {
    return (TW * TH) / 32 >= 4 ? 4 : (TW * TH) / 32;
}

struct LpConsts {
    int W, H, Wt, T;
    uint32_t n;
    int batch;
    float at, amax, teps, bg0, bg1, bg2;
};

struct LpWork {
    const int *list;
    int *counter;
    int count;
};

// staged entry: u0 = (mu_2D, sigma, -), u1..u3 = (p, q, h) x 4, u4 = (rgb, -)
struct LpStage {
    float4 *u0, *u1, *u2, *u3, *u4;
    uint32_t *id;
};

__device__ __forceinline__ void lp_stage(const float *__restrict__ sd, const uint32_t *__restrict__ vals, int e,
                                         uint32_t n, const LpStage &S, int slot) {
    const uint32_t id = __ldg(vals + e);
    if (id < n) {
        const float4 *p = reinterpret_cast<const float4 *>(sd + (size_t)id * XPR_LP_SD_FLOATS);
        S.u0[slot] = __ldg(p);
        S.u1[slot] = __ldg(p + 1);
        S.u2[slot] = __ldg(p + 2);
        S.u3[slot] = __ldg(p + 3);
        S.u4[slot] = __ldg(p + 4);
    } else {  // never blended: sigma = 0
        const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
        S.u0[slot] = z;
        S.u1[slot] = z;
        S.u2[slot] = z;
        S.u3[slot] = z;
        S.u4[slot] = z;
    }
    if (S.id) S.id[slot] = id;
}

// slab intersection at pixel centre (cx, cy); the forward and the adjoint use these operations
struct LpEval {
    float dX, dY, dt;
    int lo, hi;
};

__device__ __forceinline__ LpEval lp_eval(float cx, float cy, const float4 &u0, const float4 &u1, const float4 &u2,
                                          const float4 &u3) {
    LpEval r;
    r.dX = __fsub_rn(cx, u0.x);
    r.dY = __fsub_rn(cy, u0.y);
    const float p[4] = {u1.x, u1.w, u2.z, u3.y}, q[4] = {u1.y, u2.x, u2.w, u3.z}, h[4] = {u1.z, u2.y, u3.x, u3.w};
    float enter = __int_as_float(0xff800000), exit_ = __int_as_float(0x7f800000);
    r.lo = 0;
    r.hi = 0;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const float m = -__fmaf_rn(p[i], r.dX, __fmul_rn(q[i], r.dY));
        const float a = __fsub_rn(m, h[i]), b = __fadd_rn(m, h[i]);
        if (a > enter) {
            enter = a;
            r.lo = i;
        }
        if (b < exit_) {
            exit_ = b;
            r.hi = i;
        }
    }
    r.dt = enter < exit_ ? __fsub_rn(exit_, enter) : 0.f;
    return r;
}

// The forward needs only the chord: enter = max_i (m_i - h_i), exit = min_i (m_i + h_i), with the
// same operations as lp_eval.
__device__ __forceinline__ float lp_chord(float cx, float cy, const float4 &u0, const float4 &u1, const float4 &u2,
                                          const float4 &u3) {
    const float dX = __fsub_rn(cx, u0.x), dY = __fsub_rn(cy, u0.y);
    const float p[4] = {u1.x, u1.w, u2.z, u3.y}, q[4] = {u1.y, u2.x, u2.w, u3.z}, h[4] = {u1.z, u2.y, u3.x, u3.w};
    float enter = __int_as_float(0xff800000), exit_ = __int_as_float(0x7f800000);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const float m = -__fmaf_rn(p[i], dX, __fmul_rn(q[i], dY));
        enter = fmaxf(enter, __fsub_rn(m, h[i]));
        exit_ = fminf(exit_, __fadd_rn(m, h[i]));
    }
    return enter < exit_ ? __fsub_rn(exit_, enter) : 0.f;
}

struct LpPixFwd {
    float cy, T, r, g, b;
    int last;
    bool done;
};

template <int TW, int TH>
__device__ __forceinline__ void lp_fwd_tile(int gt, const float *__restrict__ sd, const uint32_t *__restrict__ vals,
                                            const int2 *__restrict__ ranges, const LpConsts &k,
                                            float *__restrict__ image, float *__restrict__ tfin,
                                            int *__restrict__ ncon, const LpStage &S) {
    constexpr int PX = lp_px<TW, TH>();
    constexpr int NT = TW * TH / PX, RS = TH / PX;
    static_assert(NT % 32 == 0, "a tile's block must be whole warps");
    const int v = gt / k.T, tile = gt - v * k.T;
    const int tx = tile % k.Wt, ty = tile / k.Wt;
    const int t = threadIdx.x;
    const int px = tx * TW + t % TW, py = ty * TH + t / TW;
    const int2 rg = ranges[gt];
    const float cx = (float)px + 0.5f;
    LpPixFwd P[PX];
    bool in[PX];
    bool all_done = true;
#pragma unroll
    for (int q = 0; q < PX; ++q) {
        in[q] = px < k.W && py + q * RS < k.H;
        P[q] = LpPixFwd{(float)(py + q * RS) + 0.5f, 1.f, 0.f, 0.f, 0.f, 0, !in[q]};
        all_done &= P[q].done;
    }
    for (int base = rg.x; base < rg.y; base += k.batch) {
        if (__syncthreads_and(all_done)) break;
        const int cnt = min(k.batch, rg.y - base);
        for (int e = t; e < cnt; e += NT) lp_stage(sd, vals, base + e, k.n, S, e);
        __syncthreads();
        if (!all_done) {
            for (int j = 0; j < cnt; ++j) {
                const float4 u0 = S.u0[j], u1 = S.u1[j], u2 = S.u2[j], u3 = S.u3[j], c = S.u4[j];
                const float ks = -kLog2e * u0.z;
                const int pos = base + j - rg.x;
                all_done = true;
#pragma unroll
                for (int q = 0; q < PX; ++q) {
                    LpPixFwd &p = P[q];
                    const float dt = lp_chord(cx, p.cy, u0, u1, u2, u3);
                    const float a0 = __fsub_rn(1.f, ex2_approx(__fmul_rn(ks, dt)));
                    const float al = fminf(k.amax, a0);
                    const bool live = !p.done && dt > 0.f && al >= k.at;
                    const float tt = __fmul_rn(p.T, __fsub_rn(1.f, al));
                    const bool stop = live && tt < k.teps;
                    if (live && !stop) {
                        const float w = al * p.T;
                        p.r = fmaf(c.x, w, p.r);
                        p.g = fmaf(c.y, w, p.g);
                        p.b = fmaf(c.z, w, p.b);
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
    float *img = image + (int64_t)v * 3 * HW;
#pragma unroll
    for (int q = 0; q < PX; ++q) {
        if (!in[q]) continue;
        const int64_t pix = (int64_t)(py + q * RS) * k.W + px;
        img[pix] = fmaf(P[q].T, k.bg0, P[q].r);
        img[HW + pix] = fmaf(P[q].T, k.bg1, P[q].g);
        img[2 * HW + pix] = fmaf(P[q].T, k.bg2, P[q].b);
        tfin[v * HW + pix] = P[q].T;
        ncon[v * HW + pix] = P[q].last;
    }
}

template <int TW, int TH>
__global__ void __launch_bounds__(TW *TH / lp_px<TW, TH>()) lp_render_fwd_kernel(
    const float *__restrict__ sd, const uint32_t *__restrict__ vals, const int2 *__restrict__ ranges, LpConsts k,
    float *__restrict__ image, float *__restrict__ tfin, int *__restrict__ ncon, LpWork w) {
    grid_dep_wait();
    __shared__ float4 s_u0[kLpBatch], s_u1[kLpBatch], s_u2[kLpBatch], s_u3[kLpBatch], s_u4[kLpBatch];
    const LpStage S = {s_u0, s_u1, s_u2, s_u3, s_u4, nullptr};
    if (w.list == nullptr) {
        lp_fwd_tile<TW, TH>(blockIdx.x, sd, vals, ranges, k, image, tfin, ncon, S);
        return;
    }
    __shared__ int s_item;
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) s_item = atomicAdd(w.counter, 1);
        __syncthreads();
        const int item = s_item;
        if (item >= w.count) break;
        lp_fwd_tile<TW, TH>(w.list[item], sd, vals, ranges, k, image, tfin, ncon, S);
    }
}

// Sum 32 per-lane values over the warp with 31 shuffles: at each step a lane keeps the half of its
// values selected by one bit of its lane index and sends the other half to its partner (xor 16, 8,
// 4, 2, 1).  Returns value `lane`, summed over the warp.
__device__ __forceinline__ float reduce_scatter32(const float *v, int lane) {
    float b[16];
#pragma unroll
    for (int q = 0; q < 16; ++q) {
        const bool u = lane & 16;
        b[q] = (u ? v[q + 16] : v[q]) + __shfl_xor_sync(kFullLp, u ? v[q] : v[q + 16], 16);
    }
    float c[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        const bool u = lane & 8;
        c[q] = (u ? b[q + 8] : b[q]) + __shfl_xor_sync(kFullLp, u ? b[q] : b[q + 8], 8);
    }
    float d[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const bool u = lane & 4;
        d[q] = (u ? c[q + 4] : c[q]) + __shfl_xor_sync(kFullLp, u ? c[q] : c[q + 4], 4);
    }
    float e[2];
#pragma unroll
    for (int q = 0; q < 2; ++q) {
        const bool u = lane & 2;
        e[q] = (u ? d[q + 2] : d[q]) + __shfl_xor_sync(kFullLp, u ? d[q] : d[q + 2], 2);
    }
    const bool u = lane & 1;
    return (u ? e[1] : e[0]) + __shfl_xor_sync(kFullLp, u ? e[0] : e[1], 1);
}

struct LpPixBwd {
    float cy, T, g0, g1, g2, B;  // B = g . (colour behind the current entry)
    int last;
};

// Adds pixel P's partials for the entry at list position pos (back to front) into v[32]:
//   v[k] dL/dm_k, v[4+k] dL/dm_k dX, v[8+k] dL/dm_k dY, v[12+k] dL/dh_k (k = slab), v[16] dL/dsigma,
//   v[17..19] dL/drgb.  dtau = (m_hi + h_hi) - (m_lo - h_lo).
__device__ __forceinline__ bool lp_adjoint(LpPixBwd &P, float cx, const float4 &u0, const float4 &u1,
                                           const float4 &u2, const float4 &u3, const float4 &u4, int pos,
                                           const LpConsts &k, float *v) {
    if (pos >= P.last) return false;
    const LpEval ev = lp_eval(cx, P.cy, u0, u1, u2, u3);
    if (!(ev.dt > 0.f)) return false;
    const float e = ex2_approx(__fmul_rn(-kLog2e * u0.z, ev.dt));
    const float a0 = __fsub_rn(1.f, e);
    const float al = fminf(k.amax, a0);
    if (al < k.at) return false;
    const float inv = rcp_approx(1.f - al);
    const float Ti = P.T * inv;
    const float w = al * Ti;
    v[17] = fmaf(P.g0, w, v[17]);
    v[18] = fmaf(P.g1, w, v[18]);
    v[19] = fmaf(P.g2, w, v[19]);
    const float gc = fmaf(P.g0, u4.x, fmaf(P.g1, u4.y, P.g2 * u4.z));
    const float dal = fmaf(gc, Ti, -P.B * inv);
    P.B = fmaf(gc, w, P.B);
    P.T = Ti;
    if (a0 < k.amax) {
        v[16] = fmaf(dal * ev.dt, e, v[16]);
        const float gdt = dal * u0.z * e;
#pragma unroll
        for (int s = 0; s < 4; ++s) {
            const float gm = (s == ev.hi ? gdt : 0.f) - (s == ev.lo ? gdt : 0.f);
            const float gh = (s == ev.hi ? gdt : 0.f) + (s == ev.lo ? gdt : 0.f);
            v[s] += gm;
            v[4 + s] = fmaf(gm, ev.dX, v[4 + s]);
            v[8 + s] = fmaf(gm, ev.dY, v[8 + s]);
            v[12 + s] += gh;
        }
    }
    return true;
}

template <int TW, int TH>
__device__ __forceinline__ void lp_bwd_tile(int gt, const float *__restrict__ sd, const uint32_t *__restrict__ vals,
                                            const int2 *__restrict__ ranges, const LpConsts &k,
                                            const float *__restrict__ tfin, const int *__restrict__ ncon,
                                            const float *__restrict__ dimg, float *__restrict__ d_sd,
                                            const LpStage &S, float (*s_acc)[kLpBwdBatch + 1], int *s_wmax) {
    constexpr int PX = lp_px<TW, TH>();
    constexpr int NT = TW * TH / PX, NW = NT / 32, RS = TH / PX;
    const int v = gt / k.T, tile = gt - v * k.T;
    const int tx = tile % k.Wt, ty = tile / k.Wt;
    const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
    const int px = tx * TW + t % TW, py = ty * TH + t / TW;
    const int2 rg = ranges[gt];
    const float cx = (float)px + 0.5f;
    const int64_t HW = (int64_t)k.W * k.H;
    const float *tf = tfin + v * HW;
    const int *nc = ncon + v * HW;
    const float *di = dimg + (int64_t)v * 3 * HW;
    LpPixBwd P[PX];
    int mylast = 0;
#pragma unroll
    for (int q = 0; q < PX; ++q) {
        const int y = py + q * RS;
        const bool in = px < k.W && y < k.H;
        const int64_t pix = (int64_t)y * k.W + px;
        P[q] = LpPixBwd{(float)y + 0.5f, 1.f, 0.f, 0.f, 0.f, 0.f, 0};
        if (in) {
            P[q].T = tf[pix];
            P[q].last = nc[pix];
            P[q].g0 = di[pix];
            P[q].g1 = di[HW + pix];
            P[q].g2 = di[2 * HW + pix];
        }
        P[q].B = P[q].T * fmaf(P[q].g0, k.bg0, fmaf(P[q].g1, k.bg1, P[q].g2 * k.bg2));
        mylast = max(mylast, P[q].last);
    }
    const int wlast = __reduce_max_sync(kFullLp, mylast);
    if (lane == 0) s_wmax[wid] = wlast;
    __syncthreads();
    int bmax = 0;
#pragma unroll
    for (int w = 0; w < NW; ++w) bmax = max(bmax, s_wmax[w]);
    const int batch = min(k.batch, kLpBwdBatch);
    for (int end = rg.x + bmax; end > rg.x; end -= batch) {
        const int start = max(rg.x, end - batch);
        const int cnt = end - start;
        __syncthreads();
        for (int e = t; e < cnt; e += NT) {
            lp_stage(sd, vals, start + e, k.n, S, e);
#pragma unroll
            for (int c = 0; c < 20; ++c) s_acc[c][e] = 0.f;
        }
        __syncthreads();
        for (int j = cnt - 1; j >= 0; --j) {
            const int pos = start + j - rg.x;
            if (pos >= wlast) continue;  // warp-uniform
            float vv[32];
#pragma unroll
            for (int c = 0; c < 32; ++c) vv[c] = 0.f;
            const float4 u0 = S.u0[j], u1 = S.u1[j], u2 = S.u2[j], u3 = S.u3[j], u4 = S.u4[j];
            bool hit = false;
#pragma unroll
            for (int q = 0; q < PX; ++q) hit |= lp_adjoint(P[q], cx, u0, u1, u2, u3, u4, pos, k, vv);
            if (__any_sync(kFullLp, hit)) {
                const float r = reduce_scatter32(vv, lane);
                if (lane < 20) atomicAdd(&s_acc[lane][j], r);
            }
        }
        __syncthreads();
        for (int e = t; e < cnt; e += NT) {
            float a[20];
            bool any = false;
#pragma unroll
            for (int c = 0; c < 20; ++c) {
                a[c] = s_acc[c][e];
                any |= (a[c] != 0.f);
            }
            if (any && S.id[e] < k.n) {
                const float4 u1 = S.u1[e], u2 = S.u2[e], u3 = S.u3[e];
                const float p[4] = {u1.x, u1.w, u2.z, u3.y}, q[4] = {u1.y, u2.x, u2.w, u3.z};
                // dmu_2D = sum_k (p_k, q_k) dL/dm_k;  dp_k = -sum dL/dm_k dX, dq_k likewise, dh_k
                float dmx = 0.f, dmy = 0.f;
#pragma unroll
                for (int s = 0; s < 4; ++s) {
                    dmx = fmaf(p[s], a[s], dmx);
                    dmy = fmaf(q[s], a[s], dmy);
                }
                float4 *d = reinterpret_cast<float4 *>(d_sd + (size_t)S.id[e] * XPR_LP_SD_FLOATS);
                atomicAdd(d, make_float4(dmx, dmy, a[16], 0.f));
                atomicAdd(d + 1, make_float4(-a[4], -a[8], a[12], -a[5]));
                atomicAdd(d + 2, make_float4(-a[9], a[13], -a[6], -a[10]));
                atomicAdd(d + 3, make_float4(a[14], -a[7], -a[11], a[15]));
                atomicAdd(d + 4, make_float4(a[17], a[18], a[19], 0.f));
            }
        }
    }
}

template <int TW, int TH>
__global__ void __launch_bounds__(TW *TH / lp_px<TW, TH>()) lp_render_bwd_kernel(
    const float *__restrict__ sd, const uint32_t *__restrict__ vals, const int2 *__restrict__ ranges, LpConsts k,
    const float *__restrict__ tfin, const int *__restrict__ ncon, const float *__restrict__ dimg,
    float *__restrict__ d_sd, LpWork w) {
    grid_dep_wait();
    constexpr int NW = TW * TH / lp_px<TW, TH>() / 32;
    __shared__ float4 s_u0[kLpBwdBatch], s_u1[kLpBwdBatch], s_u2[kLpBwdBatch], s_u3[kLpBwdBatch],
        s_u4[kLpBwdBatch];
    __shared__ uint32_t s_id[kLpBwdBatch];
    // rows padded by one float: the lanes adding one entry's values hit different banks
    __shared__ float s_acc[20][kLpBwdBatch + 1];
    __shared__ int s_wmax[NW];
    const LpStage S = {s_u0, s_u1, s_u2, s_u3, s_u4, s_id};
    if (w.list == nullptr) {
        lp_bwd_tile<TW, TH>(blockIdx.x, sd, vals, ranges, k, tfin, ncon, dimg, d_sd, S, s_acc, s_wmax);
        return;
    }
    __shared__ int s_item;
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) s_item = atomicAdd(w.counter, 1);
        __syncthreads();
        const int item = s_item;
        if (item >= w.count) break;
        lp_bwd_tile<TW, TH>(w.list[item], sd, vals, ranges, k, tfin, ncon, dimg, d_sd, S, s_acc, s_wmax);
    }
}

// Adjoint of one view of the LinPrim projection from d_sd (dmu_2D, dsigma, (dp, dq, dh) x 4, drgb):
//   p = n_x / n_z, q = n_y / n_z, h = 1 / |n_z|:  dn_x = dp / n_z, dn_y = dq / n_z,
//     dn_z = -(dp p + dq q + dh h) / n_z;   n_i = c0 + e1 c1 + e2 c2 (rows of A^-1);
//   dA = -A^-T dA^-1 A^-T;  A = J3 M diag(s), M = W R: dJ3 = dA (M diag(s))^T, dM = J3^T dA diag(s),
//     ds_k += sum_a dA_ak (J3 M)_ak, dR = W^T dM;  J3(m_c), mu_2D(m_c), m_c = W mu + t;
//   sigma: dsigma/do = 0.99 / ((1 - 0.99 o) 2 s_min) (0 where o is clipped), dsigma/ds_min = -sigma / s_min.
template <int DEG>
__device__ __forceinline__ void lp_adjoint_view(const Params &P, const float *shi, float *dsh, const LpGeo &G,
                                                const Cam &k, const float4 *d4, Acc<DEG> &A) {
    float D[20];
#pragma unroll
    for (int c = 0; c < 5; ++c) {
        const float4 v = __ldg(d4 + c);
        D[4 * c] = v.x;
        D[4 * c + 1] = v.y;
        D[4 * c + 2] = v.z;
        D[4 * c + 3] = v.w;
    }
    colour_adjoint<DEG>(P, shi, dsh, k, D + 16, A.mu);
    if (!G.oclip) A.o += D[2] * 0.99f / ((1.f - 0.99f * G.oc) * 2.f * G.smin);
    A.s[G.kmin] -= D[2] * G.sigma / G.smin;
    // slabs -> rows of A^-1
    float dAi[9] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        if (!(fabsf(G.n[i][2]) >= kLpEps)) continue;
        const float inz = 1.f / G.n[i][2];
        const float dp = D[4 + 3 * i], dq = D[5 + 3 * i], dh = D[6 + 3 * i];
        const float dn[3] = {dp * inz, dq * inz, -(dp * G.pqh[i][0] + dq * G.pqh[i][1] + dh * G.pqh[i][2]) * inz};
        for (int c = 0; c < 3; ++c) {
            dAi[c] += dn[c];
            dAi[3 + c] += es1(i) * dn[c];
            dAi[6 + c] += es2(i) * dn[c];
        }
    }
    // dA = -Ai^T dAi Ai^T
    float T1[9], dA[9];
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b)
            T1[3 * a + b] = G.Ai[a] * dAi[b] + G.Ai[3 + a] * dAi[3 + b] + G.Ai[6 + a] * dAi[6 + b];
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b)
            dA[3 * a + b] = -(T1[3 * a] * G.Ai[3 * b] + T1[3 * a + 1] * G.Ai[3 * b + 1] + T1[3 * a + 2] * G.Ai[3 * b + 2]);
    // A = J M diag(s)
    float dJ[9], gR[9];
    for (int a = 0; a < 3; ++a)
        for (int l = 0; l < 3; ++l)
            dJ[3 * a + l] = dA[3 * a] * G.M[3 * l] * P.s[0] + dA[3 * a + 1] * G.M[3 * l + 1] * P.s[1] +
                            dA[3 * a + 2] * G.M[3 * l + 2] * P.s[2];
    float dM[9];
    for (int l = 0; l < 3; ++l)
        for (int c = 0; c < 3; ++c)
            dM[3 * l + c] = (G.J[l] * dA[c] + G.J[3 + l] * dA[3 + c] + G.J[6 + l] * dA[6 + c]) * P.s[c];
    for (int c = 0; c < 3; ++c)
        A.s[c] += (dA[c] * G.A[c] + dA[3 + c] * G.A[3 + c] + dA[6 + c] * G.A[6 + c]) / P.s[c];
    for (int a = 0; a < 3; ++a)
        for (int c = 0; c < 3; ++c) gR[3 * a + c] = k.W[a] * dM[c] + k.W[3 + a] * dM[3 + c] + k.W[6 + a] * dM[6 + c];
    // J3(m_c) and mu_2D(m_c)
    const float x = G.mc[0], y = G.mc[1], z = G.mc[2], d = G.d;
    const float iz = 1.f / z, iz2 = iz * iz, id = 1.f / d, id3 = id * id * id;
    float gmc[3] = {0.f, 0.f, 0.f};
    gmc[2] += -k.fx * iz2 * dJ[0] - k.fy * iz2 * dJ[4];
    gmc[0] += -k.fx * iz2 * dJ[2];
    gmc[2] += 2.f * k.fx * x * iz2 * iz * dJ[2];
    gmc[1] += -k.fy * iz2 * dJ[5];
    gmc[2] += 2.f * k.fy * y * iz2 * iz * dJ[5];
    const float mdot = dJ[6] * x + dJ[7] * y + dJ[8] * z;
    gmc[0] += dJ[6] * id - x * mdot * id3;
    gmc[1] += dJ[7] * id - y * mdot * id3;
    gmc[2] += dJ[8] * id - z * mdot * id3;
    gmc[0] += D[0] * k.fx * iz;
    gmc[1] += D[1] * k.fy * iz;
    gmc[2] += -(D[0] * k.fx * x + D[1] * k.fy * y) * iz2;
    for (int j = 0; j < 3; ++j) A.mu[j] += k.W[j] * gmc[0] + k.W[3 + j] * gmc[1] + k.W[6 + j] * gmc[2];
    rotation_adjoint(G.qn, gR, A.qn);
}

template <int DEG>
__global__ void __launch_bounds__(kBwdWarps * 32, 3) lp_project_bwd_kernel(
    const float *__restrict__ mu, const float *__restrict__ scale, const float *__restrict__ quat,
    const float *__restrict__ opac, const float *__restrict__ sh, int64_t n, CamSet cs, XprConfig cfg,
    const float *__restrict__ d_sd, float *__restrict__ gmu, float *__restrict__ gscale,
    float *__restrict__ gquat, float *__restrict__ gopac, float *__restrict__ gsh) {
    grid_dep_wait();
    constexpr int KC = (DEG + 1) * (DEG + 1) * 3;
    constexpr int LD = sh_ld<DEG>();
    extern __shared__ float s_lpb[];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t base = ((int64_t)blockIdx.x * kBwdWarps + w) * 32;
    if (base >= n) return;
    const int nv = (int)min((int64_t)32, n - base);
    float *ssh = s_lpb + (size_t)w * 2 * 32 * LD;
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
            const int64_t rec_i = (int64_t)v * n + i;
            const float4 *D4 = reinterpret_cast<const float4 *>(d_sd + (size_t)rec_i * XPR_LP_SD_FLOATS);
            LpGeo G;
            lp_geometry(P, k, G);
            if (!G.front) continue;
            // the forward's visibility (box inside the grid) is reflected in d_sd: an invisible
            // record's shader data is never listed, so its gradients are zero
            lp_adjoint_view<DEG>(P, ssh + lane * LD, sdsh + lane * LD, G, k, D4, A);
            qinv = G.qinv;
            for (int j = 0; j < 4; ++j) qn[j] = G.qn[j];
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

LpConsts make_lp_consts(const XprCamera &cam, const XprConfig &cfg, int64_t n) {
    LpConsts k;
    k.n = (uint32_t)n;
    k.W = cam.width;
    k.H = cam.height;
    k.Wt = tiles_x(cam, cfg);
    k.T = tiles_x(cam, cfg) * tiles_y(cam, cfg);
    k.batch = cfg.batch_depth > 0 ? min(cfg.batch_depth, kLpBatch) : kLpBatch;
    k.at = cfg.alpha_thresh;
    k.amax = cfg.alpha_max;
    k.teps = cfg.t_eps;
    k.bg0 = cfg.bg[0];
    k.bg1 = cfg.bg[1];
    k.bg2 = cfg.bg[2];
    return k;
}

template <typename KernelT>
int lp_persistent_grid(KernelT kernel, int threads, int items) {
    int dev = 0, sms = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return items;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return items;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, 0) != cudaSuccess || per_sm < 1)
        per_sm = 1;
    return max(1, min(items, sms * per_sm));
}

#define XPR_LP_TILE_DISPATCH(TWV, THV, ...)                                                       \
    if (cfg.tile_w == 16 && cfg.tile_h == 16) { constexpr int TWV = 16, THV = 16; __VA_ARGS__; }  \
    else if (cfg.tile_w == 8 && cfg.tile_h == 8) { constexpr int TWV = 8, THV = 8; __VA_ARGS__; } \
    else if (cfg.tile_w == 16 && cfg.tile_h == 8) { constexpr int TWV = 16, THV = 8; __VA_ARGS__; } \
    else { constexpr int TWV = 8, THV = 16; __VA_ARGS__; }

}  // namespace

int launch_lp_project_fwd_views(const XprPrims &p, int64_t n, const XprCamera *cams, int n_views,
                                const XprConfig &cfg, float *rec, float *sd, int32_t *bbox, int32_t *tc,
                                int32_t *isect_count, cudaStream_t st) {
    if (n == 0 || n_views == 0) return XPR_OK;
    const int tpb = kProjWarps * 32;
    const unsigned blocks = (unsigned)((n + tpb - 1) / tpb);
    const CamSet cs = make_camset(cams, n_views);
    XPR_DEG_DISPATCH(DEG, XPR_CUDA_TRY(launch_dependent(lp_project_fwd_kernel<DEG>, dim3(blocks), dim3(tpb),
                                                        (size_t)kProjWarps * 32 * sh_ld<DEG>() * sizeof(float), st,
                                                        p.mu, p.scale, p.quat, p.opacity, p.sh, n, cs, cfg, rec, sd,
                                                        reinterpret_cast<int4 *>(bbox), tc, isect_count)));
    XPR_LAUNCH_CHECK("lp_project_fwd_kernel");
    return XPR_OK;
}

int launch_lp_project_bwd_views(const XprPrims &p, int64_t n, const XprCamera *cams, int n_views,
                                const XprConfig &cfg, const float *d_sd, const XprPrimsGrad &g, cudaStream_t st) {
    if (n == 0 || n_views == 0) return XPR_OK;
    const int tpb = kBwdWarps * 32;
    const unsigned blocks = (unsigned)((n + tpb - 1) / tpb);
    const CamSet cs = make_camset(cams, n_views);
    cudaError_t attr = cudaSuccess;
    // the shared-memory size is a constant of each instantiation, so every caller sets the same limit
    XPR_DEG_DISPATCH(DEG, {
        const size_t smem = (size_t)kBwdWarps * 2 * 32 * sh_ld<DEG>() * sizeof(float);
        attr = cudaFuncSetAttribute(lp_project_bwd_kernel<DEG>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)smem);
        if (attr == cudaSuccess)
            XPR_CUDA_TRY(launch_dependent(lp_project_bwd_kernel<DEG>, dim3(blocks), dim3(tpb), smem, st, p.mu, p.scale,
                                          p.quat, p.opacity, p.sh, n, cs, cfg, d_sd, g.mu, g.scale, g.quat, g.opacity,
                                          g.sh));
    });
    XPR_CUDA_TRY(attr);
    XPR_LAUNCH_CHECK("lp_project_bwd_kernel");
    return XPR_OK;
}

int launch_lp_bin_count(const float *sd, const int32_t *bbox, const int32_t *tc, const int32_t *order, int64_t n,
                        const XprCamera &cam, const XprConfig &cfg, int32_t *counts, cudaStream_t st) {
    if (n == 0) return XPR_OK;
    const unsigned warps = (unsigned)((n + 31) / 32);
    XPR_CUDA_TRY(launch_dependent(lp_bin_kernel<false>, dim3((warps + 7) / 8), dim3(256), 0, st, nullptr, sd,
                                  reinterpret_cast<const int4 *>(bbox), tc, order, n, make_grid(cam, cfg), counts,
                                  nullptr, nullptr, nullptr, nullptr, 0));
    XPR_LAUNCH_CHECK("lp_bin_kernel<count>");
    return XPR_OK;
}

int launch_lp_bin_emit(const float *rec, const float *sd, const int32_t *bbox, const int32_t *tc,
                       const int32_t *order, int64_t n, const XprCamera &cam, const XprConfig &cfg,
                       const int32_t *offsets, uint64_t *keys, uint32_t *tiles, uint32_t *vals, cudaStream_t st,
                       int64_t per_view) {
    if (n == 0) return XPR_OK;
    const unsigned warps = (unsigned)((n + 31) / 32);
    XPR_CUDA_TRY(launch_dependent(lp_bin_kernel<true>, dim3((warps + 7) / 8), dim3(256), 0, st, rec, sd,
                                  reinterpret_cast<const int4 *>(bbox), tc, order, n, make_grid(cam, cfg), nullptr,
                                  offsets, keys, tiles, vals, per_view));
    XPR_LAUNCH_CHECK("lp_bin_kernel<emit>");
    return XPR_OK;
}

int launch_lp_render_fwd(const float *sd, int64_t n, const uint32_t *vals, const int32_t *ranges, int n_views,
                         const XprCamera &cam, const XprConfig &cfg, float *image, float *t_final,
                         int32_t *n_contrib, const int32_t *worklist, int32_t *counter, cudaStream_t st) {
    const LpConsts k = make_lp_consts(cam, cfg, n);
    const int items = n_views * k.T;
    if (items == 0) return XPR_OK;
    const int2 *rg = reinterpret_cast<const int2 *>(ranges);
    const LpWork w = {worklist, counter, items};
    if (worklist) XPR_CUDA_TRY(cudaMemsetAsync(counter, 0, sizeof(int32_t), st));
    XPR_LP_TILE_DISPATCH(TW, TH, {
        const int threads = TW * TH / lp_px<TW, TH>();
        const int grid = worklist ? lp_persistent_grid(lp_render_fwd_kernel<TW, TH>, threads, items) : items;
        XPR_CUDA_TRY(launch_dependent(lp_render_fwd_kernel<TW, TH>, dim3(grid), dim3(threads), 0, st, sd, vals, rg, k,
                                      image, t_final, n_contrib, w));
    });
    XPR_LAUNCH_CHECK("lp_render_fwd_kernel");
    return XPR_OK;
}

int launch_lp_render_bwd(const float *sd, int64_t n, const uint32_t *vals, const int32_t *ranges, int n_views,
                         const XprCamera &cam, const XprConfig &cfg, const float *t_final, const int32_t *n_contrib,
                         const float *d_image, float *d_sd, const int32_t *worklist, int32_t *counter,
                         cudaStream_t st) {
    XPR_CUDA_TRY(cudaMemsetAsync(d_sd, 0, (size_t)n * XPR_LP_SD_FLOATS * sizeof(float), st));
    const LpConsts k = make_lp_consts(cam, cfg, n);
    const int items = n_views * k.T;
    if (items == 0) return XPR_OK;
    const int2 *rg = reinterpret_cast<const int2 *>(ranges);
    const LpWork w = {worklist, counter, items};
    if (worklist) XPR_CUDA_TRY(cudaMemsetAsync(counter, 0, sizeof(int32_t), st));
    XPR_LP_TILE_DISPATCH(TW, TH, {
        const int threads = TW * TH / lp_px<TW, TH>();
        const int grid = worklist ? lp_persistent_grid(lp_render_bwd_kernel<TW, TH>, threads, items) : items;
        XPR_CUDA_TRY(launch_dependent(lp_render_bwd_kernel<TW, TH>, dim3(grid), dim3(threads), 0, st, sd, vals, rg, k,
                                      t_final, n_contrib, d_image, d_sd, w));
    });
    XPR_LAUNCH_CHECK("lp_render_bwd_kernel");
    return XPR_OK;
}

}  // namespace xpr
