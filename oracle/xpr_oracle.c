/*
 * xpr_oracle.c -- plain FP64 CPU oracle of the 3DGS tile-splatting path.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call, link or
 * load this file; only the tests, the package entry's smoke check and the
 * benchmark's CPU-baseline leg use it.  It shares no code, header, table or
 * helper with the CUDA library.
 *
 * What it computes (citations are to the paper, arXiv 2606.11529):
 *   - projection of one 3D Gaussian (Sec. 2 "Preprocess", Listing 1 project,
 *     Appendix "Implementation of XPR-3DGS"): Sigma = R S S^T R^T, EWA
 *     footprint, conic, opacity-aware extents, tile bounding box, tile count,
 *     visibility flag, view-dependent SH colour;
 *   - the StopThePop tile cull of Listing 1 tile_cull (max response point of
 *     the tile) in FP64, its row form (per tile row, the x-extent of the
 *     ellipse within the row's strip) in FP64, and the row form in an
 *     exact-FP32 version whose operation order is fixed and FMA-free
 *     (decisions taken in the kernels' precision);
 *   - replicate / assign-tile-ID / sort / segment bounds of Sec. 4.2;
 *   - front-to-back alpha compositing c = sum c_i a_i T_i (Sec. 2 "Shader",
 *     Algorithm 1) with the evaluate of Listing 1, as a brute-force
 *     all-primitives walk per pixel (the evaluate_full view of Sec. 3.1) and
 *     as a per-tile walk over given lists;
 *   - the analytic adjoint of compositing and of the projection, written from
 *     the definitions (explicit suffix sums, explicit matrix-inverse
 *     derivative), for checking the hand-written CUDA backward.
 * Readings of points the paper leaves open (dilation 0.3 and Jacobian clamp
 * 1.3, alpha clamp 0.99, T_eps 1e-4 tested before accumulating, raw pixel
 * coordinates for 3DGS, extents sqrt(2 ln(o/a_t) Sigma_xx), SH convention)
 * are taken as the config values passed in.
 *
 * Camera array (19 doubles): W, H, fx, fy, cx, cy, V[12] (world->camera 3x4
 * row-major), z_near.  Config array (11 doubles): tile_w, tile_h, alpha_t,
 * alpha_max, t_eps, dilation, clip, sh_degree, bg_r, bg_g, bg_b.
 *
 * Record layout (12 per primitive): mx, my, c00, c01, c11, o, r, g, b,
 * depth, ln_thr, visible.  bbox (4 ints): xmin, ymin, xmax, ymax (tiles,
 * half-open).
 *
 * Build: gcc -O2 -ffp-contract=off -fopenmp -shared -fPIC (no fast-math: the
 * exact-FP32 cull relies on IEEE single rounding of every operation).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define O_PI 3.14159265358979323846

typedef struct {
    int W, H;
    double fx, fy, cx, cy;
    double V[12];
    double z_near;
    int model;    /* 0 pinhole, 1 fisheye (3DGUT) */
    double k[4];  /* fisheye: theta_d = theta (1 + k1 theta^2 + k2 theta^4 + k3 theta^6 + k4 theta^8) */
} ocam;

typedef struct {
    int tw, th;
    double at, amax, teps, dil, clip;
    int deg;
    double bg[3];
    int method; /* 0 = 3DGS (EWA), 1 = 3DGUT (unscented transform, ray evaluation) */
} ocfg;

static ocam read_cam(const double *c) {
    ocam k;
    k.W = (int)c[0];
    k.H = (int)c[1];
    k.fx = c[2];
    k.fy = c[3];
    k.cx = c[4];
    k.cy = c[5];
    for (int i = 0; i < 12; ++i) k.V[i] = c[6 + i];
    k.z_near = c[18];
    k.model = (int)c[19];
    for (int i = 0; i < 4; ++i) k.k[i] = c[20 + i];
    return k;
}

static ocfg read_cfg(const double *c) {
    ocfg g;
    g.tw = (int)c[0];
    g.th = (int)c[1];
    g.at = c[2];
    g.amax = c[3];
    g.teps = c[4];
    g.dil = c[5];
    g.clip = c[6];
    g.deg = (int)c[7];
    g.bg[0] = c[8];
    g.bg[1] = c[9];
    g.bg[2] = c[10];
    g.method = (int)c[11];
    return g;
}

/* ------------------------------------------------------------------------ */
/* Real spherical harmonics (Condon-Shortley phase), general degree.         */
/* For a unit direction (x, y, z):                                           */
/*   Y_l^0  = K_l^0 Q_l^0(z)                                                 */
/*   Y_l^m  = sqrt2 K_l^m Q_l^m(z) Re((x+iy)^m)      m > 0                   */
/*   Y_l^-m = sqrt2 K_l^m Q_l^m(z) Im((x+iy)^m)      m > 0                   */
/* with Q_l^m(z) = P_l^m(z) / (1-z^2)^{m/2} (associated Legendre with the    */
/* Condon-Shortley phase, divided by sin^m theta) and                        */
/* K_l^m = sqrt((2l+1)/(4 pi) (l-m)!/(l+m)!).  Index k = l^2 + l + m.        */
/* ------------------------------------------------------------------------ */

static double factorial(int n) {
    double f = 1.0;
    for (int i = 2; i <= n; ++i) f *= (double)i;
    return f;
}

/* Q[l][m] for l, m <= deg+1 via the standard three-term recurrence. */
static void legendre_q(int lmax, double z, double Q[6][6]) {
    for (int m = 0; m <= lmax; ++m) {
        /* Q_m^m = (-1)^m (2m-1)!! */
        double qmm = 1.0;
        for (int i = 1; i <= m; ++i) qmm *= -(2.0 * i - 1.0);
        Q[m][m] = qmm;
        if (m + 1 <= lmax) Q[m + 1][m] = z * (2.0 * m + 1.0) * qmm;
        for (int l = m + 2; l <= lmax; ++l)
            Q[l][m] = ((2.0 * l - 1.0) * z * Q[l - 1][m] - (double)(l + m - 1) * Q[l - 2][m]) / (double)(l - m);
    }
}

/* Y[k] and, if grad != NULL, dY/d(x,y,z) as [k][3] for the polynomial
 * extension above (the caller projects onto the sphere's tangent plane). */
void oracle_sh_basis(int deg, const double *d, double *Y, double *grad) {
    double x = d[0], y = d[1], z = d[2];
    double Q[6][6];
    memset(Q, 0, sizeof(Q));
    legendre_q(deg + 1, z, Q);
    /* powers (x+iy)^m = re[m] + i im[m] */
    double re[6], im[6];
    re[0] = 1.0;
    im[0] = 0.0;
    for (int m = 1; m <= deg + 1; ++m) {
        re[m] = re[m - 1] * x - im[m - 1] * y;
        im[m] = re[m - 1] * y + im[m - 1] * x;
    }
    for (int l = 0; l <= deg; ++l) {
        for (int m = 0; m <= l; ++m) {
            double K = sqrt((2.0 * l + 1.0) / (4.0 * O_PI) * factorial(l - m) / factorial(l + m));
            /* dQ_l^m/dz = -Q_l^{m+1} (Q_l^{l+1} = 0) */
            double q = Q[l][m];
            double dq = (m + 1 <= l) ? -Q[l][m + 1] : 0.0;
            if (m == 0) {
                int k = l * l + l;
                Y[k] = K * q;
                if (grad) {
                    grad[3 * k + 0] = 0.0;
                    grad[3 * k + 1] = 0.0;
                    grad[3 * k + 2] = K * dq;
                }
            } else {
                double s2k = sqrt(2.0) * K;
                int kp = l * l + l + m, kn = l * l + l - m;
                Y[kp] = s2k * q * re[m];
                Y[kn] = s2k * q * im[m];
                if (grad) {
                    /* d/dx (x+iy)^m = m (x+iy)^{m-1};  d/dy = i m (x+iy)^{m-1} */
                    grad[3 * kp + 0] = s2k * q * m * re[m - 1];
                    grad[3 * kp + 1] = s2k * q * (-(double)m * im[m - 1]);
                    grad[3 * kp + 2] = s2k * dq * re[m];
                    grad[3 * kn + 0] = s2k * q * m * im[m - 1];
                    grad[3 * kn + 1] = s2k * q * m * re[m - 1];
                    grad[3 * kn + 2] = s2k * dq * im[m];
                }
            }
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Projection of one primitive (Listing 1 project; Sec. 2 Preprocess).       */
/* ------------------------------------------------------------------------ */

typedef struct {
    double qn[4], qnorm;
    double R[9];      /* primitive rotation */
    double Sig[9];    /* 3D covariance */
    double mc[3];     /* camera-space mean */
    double ux, uy;    /* clamped x/z, y/z used by the Jacobian */
    int clx, cly;     /* 1 if clamped */
    double J[6];      /* 2x3 */
    double Tm[6];     /* J * W (2x3) */
    double cov[3];    /* a, b, c of Sigma_2D (dilated) */
    double cabs[3];   /* the same sums over absolute values (|T| |Sigma| |T|^T + dilation) */
    double det;
    double conic[3];
    double mu2d[2];
    double ln_thr, ex, ey;
    double pre[4];    /* values before floor: (mx-ex)/w, (my-ey)/h, (mx+ex)/w, (my+ey)/h */
    int bbox[4], tc, visible;
    double dir[3], vlen; /* unit view direction and |mu - campos| */
    double raw[3], rgb[3];
} oproj;

static void quat_rot(const double *q, double *qn, double *qnorm, double *R) {
    double n = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
    *qnorm = n;
    double w = q[0] / n, x = q[1] / n, y = q[2] / n, z = q[3] / n;
    qn[0] = w;
    qn[1] = x;
    qn[2] = y;
    qn[3] = z;
    R[0] = 1.0 - 2.0 * (y * y + z * z);
    R[1] = 2.0 * (x * y - w * z);
    R[2] = 2.0 * (x * z + w * y);
    R[3] = 2.0 * (x * y + w * z);
    R[4] = 1.0 - 2.0 * (x * x + z * z);
    R[5] = 2.0 * (y * z - w * x);
    R[6] = 2.0 * (x * z - w * y);
    R[7] = 2.0 * (y * z + w * x);
    R[8] = 1.0 - 2.0 * (x * x + y * y);
}

static double clampd(double v, double lo, double hi) { return v < lo ? lo : (v > hi ? hi : v); }

static void project_one(const double *mu, const double *s, const double *q, double o, const double *sh,
                        const ocam *cam, const ocfg *cfg, oproj *P) {
    memset(P, 0, sizeof(*P));
    const double *V = cam->V;
    /* world -> camera */
    for (int i = 0; i < 3; ++i) P->mc[i] = V[4 * i] * mu[0] + V[4 * i + 1] * mu[1] + V[4 * i + 2] * mu[2] + V[4 * i + 3];
    double x = P->mc[0], y = P->mc[1], z = P->mc[2];

    /* Sigma = R S S^T R^T (Sec. 2) */
    quat_rot(q, P->qn, &P->qnorm, P->R);
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double acc = 0.0;
            for (int k = 0; k < 3; ++k) acc += P->R[3 * i + k] * s[k] * s[k] * P->R[3 * j + k];
            P->Sig[3 * i + j] = acc;
        }

    /* view direction and SH colour, rgb = max(0, sum sh_k Y_k(d) + 0.5) */
    double cp[3]; /* camera position = -R_v^T t */
    for (int i = 0; i < 3; ++i) cp[i] = -(V[i] * V[3] + V[4 + i] * V[7] + V[8 + i] * V[11]);
    double v[3] = {mu[0] - cp[0], mu[1] - cp[1], mu[2] - cp[2]};
    P->vlen = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
    for (int i = 0; i < 3; ++i) P->dir[i] = v[i] / P->vlen;
    int K = (cfg->deg + 1) * (cfg->deg + 1);
    double Y[16];
    oracle_sh_basis(cfg->deg, P->dir, Y, NULL);
    for (int c = 0; c < 3; ++c) {
        double acc = 0.0;
        for (int k = 0; k < K; ++k) acc += sh[3 * k + c] * Y[k];
        P->raw[c] = acc + 0.5;
        P->rgb[c] = P->raw[c] > 0.0 ? P->raw[c] : 0.0;
    }

    if (!(z > cam->z_near)) { /* behind the near plane: nothing else is defined */
        P->visible = 0;
        return;
    }

    /* EWA: J = d(pixel)/d(camera point), x/z and y/z clamped to 1.3 x half-fov */
    double limx = cfg->clip * (0.5 * cam->W / cam->fx);
    double limy = cfg->clip * (0.5 * cam->H / cam->fy);
    double rx = x / z, ry = y / z;
    P->ux = clampd(rx, -limx, limx);
    P->uy = clampd(ry, -limy, limy);
    P->clx = (rx < -limx || rx > limx);
    P->cly = (ry < -limy || ry > limy);
    P->J[0] = cam->fx / z;
    P->J[1] = 0.0;
    P->J[2] = -cam->fx * P->ux / z;
    P->J[3] = 0.0;
    P->J[4] = cam->fy / z;
    P->J[5] = -cam->fy * P->uy / z;
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 3; ++j) {
            double acc = 0.0;
            for (int k = 0; k < 3; ++k) acc += P->J[3 * i + k] * V[4 * k + j];
            P->Tm[3 * i + j] = acc;
        }
    double C2[4], C2a[4];
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 2; ++j) {
            double acc = 0.0, aacc = 0.0;
            for (int k = 0; k < 3; ++k)
                for (int l = 0; l < 3; ++l) {
                    acc += P->Tm[3 * i + k] * P->Sig[3 * k + l] * P->Tm[3 * j + l];
                    aacc += fabs(P->Tm[3 * i + k] * P->Sig[3 * k + l] * P->Tm[3 * j + l]);
                }
            C2[2 * i + j] = acc;
            C2a[2 * i + j] = aacc;
        }
    P->cabs[0] = C2a[0] + cfg->dil;
    P->cabs[1] = 0.5 * (C2a[1] + C2a[2]);
    P->cabs[2] = C2a[3] + cfg->dil;
    P->cov[0] = C2[0] + cfg->dil;
    P->cov[1] = 0.5 * (C2[1] + C2[2]);
    P->cov[2] = C2[3] + cfg->dil;
    P->det = P->cov[0] * P->cov[2] - P->cov[1] * P->cov[1];
    P->mu2d[0] = cam->fx * rx + cam->cx;
    P->mu2d[1] = cam->fy * ry + cam->cy;
    if (!(P->det > 0.0) || !(o >= cfg->at)) {
        P->visible = 0;
        return;
    }
    P->conic[0] = P->cov[2] / P->det;
    P->conic[1] = -P->cov[1] / P->det;
    P->conic[2] = P->cov[0] / P->det;

    /* opacity-aware extents of {alpha >= alpha_t}: |dx| <= sqrt(2 ln(o/a_t) Sigma_xx) */
    P->ln_thr = log(o / cfg->at);
    P->ex = sqrt(2.0 * P->ln_thr * P->cov[0]);
    P->ey = sqrt(2.0 * P->ln_thr * P->cov[2]);
    double r = P->ex > P->ey ? P->ex : P->ey;

    /* half-open tile-space bounding box (Sec. 4.2) */
    int Wt = (cam->W + cfg->tw - 1) / cfg->tw, Ht = (cam->H + cfg->th - 1) / cfg->th;
    P->pre[0] = (P->mu2d[0] - P->ex) / cfg->tw;
    P->pre[1] = (P->mu2d[1] - P->ey) / cfg->th;
    P->pre[2] = (P->mu2d[0] + P->ex) / cfg->tw;
    P->pre[3] = (P->mu2d[1] + P->ey) / cfg->th;
    P->bbox[0] = (int)clampd(floor(P->pre[0]), 0.0, (double)Wt);
    P->bbox[1] = (int)clampd(floor(P->pre[1]), 0.0, (double)Ht);
    P->bbox[2] = (int)clampd(floor(P->pre[2]) + 1.0, 0.0, (double)Wt);
    P->bbox[3] = (int)clampd(floor(P->pre[3]) + 1.0, 0.0, (double)Ht);
    int tc = (P->bbox[2] - P->bbox[0]) * (P->bbox[3] - P->bbox[1]);
    /* visible = det>0 & o>=a_t & r>0 & tc>0 & z>z_near (Listing 1) */
    P->visible = (r > 0.0) && (tc > 0);
    P->tc = P->visible ? tc : 0;
    if (!P->visible) memset(P->bbox, 0, sizeof(P->bbox));
}

static void write_rec(const oproj *P, double o, double *rec) {
    memset(rec, 0, 12 * sizeof(double));
    rec[9] = P->mc[2];
    if (!P->visible) return;
    rec[0] = P->mu2d[0];
    rec[1] = P->mu2d[1];
    rec[2] = P->conic[0];
    rec[3] = P->conic[1];
    rec[4] = P->conic[2];
    rec[5] = o;
    rec[6] = P->rgb[0];
    rec[7] = P->rgb[1];
    rec[8] = P->rgb[2];
    rec[10] = P->ln_thr;
    rec[11] = 1.0;
}

/* Projection of n primitives.  rec[n*12], bbox[n*4], tc[n]; pre[n*4] and
 * cov[n*3] (dilated Sigma_2D) may be NULL. */
void oracle_project(int64_t n, const double *mu, const double *scale, const double *quat, const double *opac,
                    const double *sh, const double *camv, const double *cfgv, double *rec, int32_t *bbox,
                    int32_t *tc, double *pre, double *cov) {
    ocam cam = read_cam(camv);
    ocfg cfg = read_cfg(cfgv);
    int K = (cfg.deg + 1) * (cfg.deg + 1);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        oproj P;
        project_one(mu + 3 * i, scale + 3 * i, quat + 4 * i, opac[i], sh + (int64_t)3 * K * i, &cam, &cfg, &P);
        write_rec(&P, opac[i], rec + 12 * i);
        for (int j = 0; j < 4; ++j) bbox[4 * i + j] = P.bbox[j];
        tc[i] = P.tc;
        if (pre)
            for (int j = 0; j < 4; ++j) pre[4 * i + j] = P.visible ? P.pre[j] : 0.0;
        if (cov)
            for (int j = 0; j < 3; ++j) cov[3 * i + j] = P.cov[j];
    }
}

/* Scales of a float32 projection's rounding, per primitive (test infrastructure for the ambiguity
 * band of the compositing walk; no part of the method).  unc[n*5] = (m, k, sa, sb, sc):
 *   m  = the centre's rounding model in pixels, e = 2^-24:
 *        e (3 |f x/z| + |mu_2D| + 3 f (s_x + |x/z| s_z) / z), s_i = sum_j |V_ij mu_j| + |V_i3|,
 *        the larger of the x and y expressions (m_c = W mu + t carries ~3 e s_i per component,
 *        x/z two roundings more, f x/z + c one more relative to |mu_2D|);
 *   k  = a c / (a c - b^2) of Sigma_2D: the relative precision the 2x2 inverse loses;
 *   sa, sb, sc = |T| |Sigma| |T|^T + dilation I (T = J W): the scale of the rounding of the
 *        Sigma_2D entries, whose first-order effect on power = -d^T Sigma_2D^-1 d / 2 is
 *        g^T dSigma_2D g / 2 with g = conic d. */
void oracle_project_unc(int64_t n, const double *mu, const double *scale, const double *quat, const double *opac,
                        const double *sh, const double *camv, const double *cfgv, double *unc) {
    ocam cam = read_cam(camv);
    ocfg cfg = read_cfg(cfgv);
    int K = (cfg.deg + 1) * (cfg.deg + 1);
    const double e = 1.0 / 16777216.0;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        oproj P;
        project_one(mu + 3 * i, scale + 3 * i, quat + 4 * i, opac[i], sh + (int64_t)3 * K * i, &cam, &cfg, &P);
        double *u = unc + 5 * i;
        for (int j = 0; j < 5; ++j) u[j] = 0.0;
        if (!P.visible) continue;
        double sv[3];
        for (int r = 0; r < 3; ++r) {
            sv[r] = fabs(cam.V[4 * r + 3]);
            for (int j = 0; j < 3; ++j) sv[r] += fabs(cam.V[4 * r + j] * mu[3 * i + j]);
        }
        double z = P.mc[2], rx = P.mc[0] / z, ry = P.mc[1] / z;
        double mx = e * (3.0 * fabs(cam.fx * rx) + fabs(P.mu2d[0]) + 3.0 * cam.fx * (sv[0] + fabs(rx) * sv[2]) / z);
        double my = e * (3.0 * fabs(cam.fy * ry) + fabs(P.mu2d[1]) + 3.0 * cam.fy * (sv[1] + fabs(ry) * sv[2]) / z);
        u[0] = mx > my ? mx : my;
        u[1] = P.cov[0] * P.cov[2] / P.det;
        u[2] = P.cabs[0];
        u[3] = P.cabs[1];
        u[4] = P.cabs[2];
    }
}

/* ------------------------------------------------------------------------ */
/* Depth sort key (Sec. 4.2 sorts by tile, then depth; reading of the tie     */
/* order: (tile, float32 bits of the depth, primitive index)).  The order is */
/* an integer decision, so it is taken in the kernels' precision from the    */
/* float32 inputs, with every operation rounded to float32 in a fixed order  */
/* and no fused multiply-add:                                                */
/*   m_c,i = ((V_i0 x + V_i1 y) + V_i2 z) + V_i3                             */
/*   key = m_c,2 (camera z; 3DGS and 3DGUT), or                               */
/*   key = sqrt((x_c x_c + y_c y_c) + z_c z_c)  (LinPrim's Euclidean depth).  */
/* ------------------------------------------------------------------------ */

static float cam_axis32(const ocam *cam, int i, const float *m) {
    float a = (float)cam->V[4 * i] * m[0];
    float b = (float)cam->V[4 * i + 1] * m[1];
    float c = (float)cam->V[4 * i + 2] * m[2];
    float s = a + b;
    s = s + c;
    return s + (float)cam->V[4 * i + 3];
}

void oracle_depth_keys(int64_t n, const double *mu, const double *camv, int euclid, float *key) {
    ocam cam = read_cam(camv);
    for (int64_t i = 0; i < n; ++i) {
        float m[3] = {(float)mu[3 * i], (float)mu[3 * i + 1], (float)mu[3 * i + 2]};
        float z = cam_axis32(&cam, 2, m);
        if (euclid) {
            float x = cam_axis32(&cam, 0, m), y = cam_axis32(&cam, 1, m);
            float xx = x * x, yy = y * y, zz = z * z;
            float s = xx + yy;
            s = s + zz;
            z = sqrtf(s);
        }
        key[i] = z;
    }
}

/* ------------------------------------------------------------------------ */
/* StopThePop tile cull (Listing 1 tile_cull; Appendix 3DGS implementation). */
/* The response o exp(-q/2), q = d^T conic d, d = mu - p, is largest at the  */
/* point p of the tile closest to mu in the conic metric: mu itself when mu  */
/* lies in the tile, else the best point of the (at most two) tile edges     */
/* that face mu; on an edge the 1-D quadratic is minimised in closed form    */
/* and clamped to the edge.  Keep iff q/2 <= ln(o / alpha_t).               */
/* Tile bounds are inclusive pixel coordinates:                              */
/*   x0 = tx w, x1 = min(tx w + w - 1, W - 1)  (same in y).                  */
/* ------------------------------------------------------------------------ */

static int cull_f64(double mx, double my, double c0, double c1, double c2, double lt, double x0, double y0,
                    double x1, double y1) {
    int outx = (mx < x0) || (mx > x1);
    int outy = (my < y0) || (my > y1);
    if (!outx && !outy) return 0.0 <= lt;
    double best = INFINITY;
    if (outx) {
        double ex = mx < x0 ? x0 : x1;
        double dx = mx - ex;
        double ys = clampd(my + c1 * dx / c2, y0, y1);
        double dy = my - ys;
        double p = 0.5 * (c0 * dx * dx + 2.0 * c1 * dx * dy + c2 * dy * dy);
        if (p < best) best = p;
    }
    if (outy) {
        double ey = my < y0 ? y0 : y1;
        double dy = my - ey;
        double xs = clampd(mx + c1 * dy / c0, x0, x1);
        double dx = mx - xs;
        double p = 0.5 * (c0 * dx * dx + 2.0 * c1 * dx * dy + c2 * dy * dy);
        if (p < best) best = p;
    }
    return best <= lt;
}

/* Row form of the same cull.  Inside one tile row (pixel rows [y0, y1]) the
 * largest response over a tile reaches alpha_t iff the tile's pixel columns
 * [x0, x1] meet S = {x : min over y in [y0, y1] of q(x, y) <= 2 ln_thr}, the
 * x-extent of E ∩ strip with E = {q <= T}, T = 2 ln_thr.  E ∩ strip is
 * convex, so S is one interval [xa, xb]: xa (xb) is the least (greatest) x
 * among the leftmost (rightmost) point of E when its y lies in the strip and
 * the crossings of the boundary of E with the lines y = y0 and y = y1.  With
 * conic [[a, b], [b, c]], det = ac - b^2: the leftmost / rightmost points are
 * (mx -/+ ex, my +/- sb), ex = sqrt(T c / det), sb = b sqrt(T / (c det)); the
 * crossings with y = Y are x = mx + (-b dY -/+ sqrt(a T - det dY^2)) / a,
 * dY = Y - my.  In exact arithmetic this keeps exactly the tiles the
 * per-tile minimum keeps; it costs one evaluation per row instead of one per
 * tile.  Returns 0 when the strip misses E. */
static int row_span_f64(double mx, double my, double a, double b, double c, double lt, double y0, double y1,
                        double *xa, double *xb) {
    double T = 2.0 * lt;
    if (!(T >= 0.0)) return 0;
    double det = a * c - b * b;
    double ex = sqrt(T * c / det), sb = b * sqrt(T / (c * det));
    double lo = INFINITY, hi = -INFINITY;
    double yl = my + sb, yr = my - sb;
    if (yl >= y0 && yl <= y1) lo = mx - ex;
    if (yr >= y0 && yr <= y1) hi = mx + ex;
    double ys[2] = {y0, y1};
    for (int k = 0; k < 2; ++k) {
        double dY = ys[k] - my;
        double disc = a * T - det * dY * dY;
        if (disc >= 0.0) {
            double r = sqrt(disc);
            double xl = mx + (-b * dY - r) / a, xr = mx + (-b * dY + r) / a;
            if (xl < lo) lo = xl;
            if (xr > hi) hi = xr;
        }
    }
    if (!(lo <= hi)) return 0;
    *xa = lo;
    *xb = hi;
    return 1;
}

/* Per-tile decision of the row form in FP64: keep iff [x0, x1] meets [xa, xb]. */
static int cull_row_f64(double mx, double my, double c0, double c1, double c2, double lt, double x0, double y0,
                        double x1, double y1) {
    double xa, xb;
    if (!row_span_f64(mx, my, c0, c1, c2, lt, y0, y1, &xa, &xb)) return 0;
    return x1 >= xa && x0 <= xb;
}

/* The row form in IEEE single precision, one rounding per operation in this
 * exact order, no FMA (the CUDA kernels take the decision in FP32 with the
 * same sequence of correctly rounded operations: +, -, *, /, sqrt, and the
 * correctly rounded reciprocal 1/a).  Per primitive: */
typedef struct {
    float mx, my, b, det, aT, ia, ex, yl, yr;
    int ok;
} rowcull32;

static rowcull32 rowcull32_make(const float *R) {
    rowcull32 r;
    float a = R[2], b = R[3], c = R[4], lt = R[10];
    float T = lt + lt;
    r.mx = R[0];
    r.my = R[1];
    r.b = b;
    r.ok = T >= 0.0f;
    float ac = a * c, bb = b * b;
    r.det = ac - bb;
    r.aT = a * T;
    r.ia = 1.0f / a;
    float e1 = T * c;
    float e2 = e1 / r.det;
    r.ex = sqrtf(e2);
    float s1 = c * r.det;
    float s2 = T / s1;
    float s3 = sqrtf(s2);
    float sb = b * s3;
    r.yl = r.my + sb;
    r.yr = r.my - sb;
    return r;
}

/* Kept tile columns [*ka, *kb] of tile row ty (pixel rows y0..y1); 0 if none.
 * Tile k spans pixel columns [k w, k w + w - 1] (the last one clamped to
 * W - 1): k w + w - 1 >= xa  <=>  k >= ceil((xa + 1) / w) - 1, and k w <= xb
 * <=> k <= floor(xb / w); a span starting right of the image or ending left
 * of it keeps nothing. */
static int row_tiles_f32(const rowcull32 *r, float y0, float y1, int w, int W, int ext, int *ka, int *kb) {
    if (!r->ok) return 0;
    float lo = INFINITY, hi = -INFINITY;
    if (r->yl >= y0 && r->yl <= y1) lo = r->mx - r->ex;
    if (r->yr >= y0 && r->yr <= y1) hi = r->mx + r->ex;
    float ys[2] = {y0, y1};
    for (int k = 0; k < 2; ++k) {
        float dY = ys[k] - r->my;
        float q1 = r->det * dY;
        float q2 = q1 * dY;
        float disc = r->aT - q2;
        if (disc >= 0.0f) {
            float rt = sqrtf(disc);
            float m = r->b * dY;
            float nm = -m;
            float ul = nm - rt, ur = nm + rt;
            float xl = ul * r->ia, xr = ur * r->ia;
            xl = r->mx + xl;
            xr = r->mx + xr;
            lo = fminf(lo, xl);
            hi = fmaxf(hi, xr);
        }
    }
    if (!(lo <= hi)) return 0;
    if (lo > (float)(W - 1 + ext) || hi < 0.0f) return 0;
    float iw = 1.0f / (float)w;
    float t = lo + (float)(1 - ext); /* tile k is kept iff k w + w - 1 + ext >= xa */
    t = t * iw;
    float u = hi * iw;
    t = fmaxf(t, -1.0f);
    u = fminf(u, (float)(W / w + 2));
    *ka = (int)ceilf(t) - 1;
    *kb = (int)floorf(u);
    return *ka <= *kb;
}

/* 3DGUT (method 1) extends the max bounds by one: its pixel centres sit at +0.5, so tile
 * [x0, x1] of pixel indices covers [x0, x1 + 1] in the continuous coordinates of its means. */
static void tile_bounds(int tx, int ty, const ocam *cam, const ocfg *cfg, double *b) {
    int x0 = tx * cfg->tw, y0 = ty * cfg->th;
    int x1 = x0 + cfg->tw - 1, y1 = y0 + cfg->th - 1;
    if (x1 > cam->W - 1) x1 = cam->W - 1;
    if (y1 > cam->H - 1) y1 = cam->H - 1;
    x1 += cfg->method == 1;
    y1 += cfg->method == 1;
    b[0] = x0;
    b[1] = y0;
    b[2] = x1;
    b[3] = y1;
}

/* Exposed for the dense-sampling pin of the cull (FP64 form). form 0: the
 * per-tile minimum; 1: the row form (FP64); 2: the row form in FP32 on the
 * float-rounded record (the kernels' decision). */
int oracle_cull_one(const double *rec, int tx, int ty, const double *camv, const double *cfgv, int form) {
    ocam cam = read_cam(camv);
    ocfg cfg = read_cfg(cfgv);
    double b[4];
    tile_bounds(tx, ty, &cam, &cfg, b);
    if (form == 1) return cull_row_f64(rec[0], rec[1], rec[2], rec[3], rec[4], rec[10], b[0], b[1], b[2], b[3]);
    if (form == 2) {
        float R[12];
        for (int k = 0; k < 12; ++k) R[k] = (float)rec[k];
        rowcull32 rc = rowcull32_make(R);
        int ka, kb;
        if (!row_tiles_f32(&rc, (float)b[1], (float)b[3], cfg.tw, cam.W, cfg.method == 1, &ka, &kb)) return 0;
        return tx >= ka && tx <= kb;
    }
    return cull_f64(rec[0], rec[1], rec[2], rec[3], rec[4], rec[10], b[0], b[1], b[2], b[3]);
}

static uint32_t f32_bits(float f) {
    uint32_t u;
    memcpy(&u, &f, 4);
    return u;
}

/* Replicate + assign tile ID + cull (Sec. 4.2).  For every primitive in
 * index order and every slot r in 0..tc-1 of its bounding box (row-major:
 * x = xmin + r mod w_i, y = ymin + r div w_i, t = y W' + x), keep the pair if
 * the cull passes and emit key = (t << 32) | bits(float(depth)), val = i.
 * exact32 != 0: rec32 (float records) with the FP32 cull and the records'
 * own depths; else rec64 with the FP64 cull and the depth keys key[n]
 * (oracle_depth_keys; NULL = the FP64 depth rounded to float32).  order (may be NULL = index order) gives the order in which the
 * primitives are visited; counts[n] receives the surviving count per visited
 * position.  keys and vals may be NULL (count only).  Returns the total. */
int64_t oracle_bin(int64_t n, const double *rec64, const float *rec32, const float *key, const int32_t *bbox,
                   const double *camv, const double *cfgv, int exact32, const int64_t *order, int32_t *counts,
                   uint64_t *keys, uint32_t *vals) {
    ocam cam = read_cam(camv);
    ocfg cfg = read_cfg(cfgv);
    int Wt = (cam.W + cfg.tw - 1) / cfg.tw;
    int64_t total = 0;
    /* primitives are visited in the given order (identity when NULL); counts are per position */
    for (int64_t pos = 0; pos < n; ++pos) {
        int64_t i = order ? order[pos] : pos;
        const int32_t *bb = bbox + 4 * i;
        int w = bb[2] - bb[0], h = bb[3] - bb[1];
        int tc = (w > 0 && h > 0) ? w * h : 0;
        int cnt = 0;
        rowcull32 rc;
        if (exact32 && tc > 0) rc = rowcull32_make(rec32 + 12 * i);
        int row_ty = -1, ka = 0, kb = -1;
        for (int r = 0; r < tc; ++r) {
            int tx = bb[0] + r % w, ty = bb[1] + r / w;
            double b[4];
            tile_bounds(tx, ty, &cam, &cfg, b);
            int keep;
            float depth32;
            if (exact32) {
                const float *R = rec32 + 12 * i;
                if (ty != row_ty) {  /* one span per tile row */
                    row_ty = ty;
                    if (!row_tiles_f32(&rc, (float)b[1], (float)b[3], cfg.tw, cam.W, cfg.method == 1, &ka, &kb)) {
                        ka = 0;
                        kb = -1;
                    }
                }
                keep = tx >= ka && tx <= kb;
                depth32 = R[9];
            } else {
                const double *R = rec64 + 12 * i;
                keep = cull_f64(R[0], R[1], R[2], R[3], R[4], R[10], b[0], b[1], b[2], b[3]);
                depth32 = key ? key[i] : (float)R[9];
            }
            if (!keep) continue;
            if (keys) {
                keys[total] = ((uint64_t)(uint32_t)(ty * Wt + tx) << 32) | (uint64_t)f32_bits(depth32);
                vals[total] = (uint32_t)i;
            }
            ++total;
            ++cnt;
        }
        if (counts) counts[pos] = cnt;
    }
    return total;
}

/* Sort (key, val) pairs ascending by key then val and find per-tile
 * segment bounds [start, end) (Sec. 4.2, "Sort and identify bounds").
 * ranges[n_tiles*2] is fully written (empty tiles get [0,0)). */
typedef struct {
    uint64_t k;
    uint32_t v;
} kv_t;

static int kv_cmp(const void *a, const void *b) {
    const kv_t *x = (const kv_t *)a, *y = (const kv_t *)b;
    if (x->k != y->k) return x->k < y->k ? -1 : 1;
    if (x->v != y->v) return x->v < y->v ? -1 : 1;
    return 0;
}

void oracle_sort(int64_t m, uint64_t *keys, uint32_t *vals, int64_t n_tiles, int32_t *ranges) {
    kv_t *a = (kv_t *)malloc((size_t)(m > 0 ? m : 1) * sizeof(kv_t));
    for (int64_t i = 0; i < m; ++i) {
        a[i].k = keys[i];
        a[i].v = vals[i];
    }
    qsort(a, (size_t)m, sizeof(kv_t), kv_cmp);
    for (int64_t i = 0; i < m; ++i) {
        keys[i] = a[i].k;
        vals[i] = a[i].v;
    }
    free(a);
    for (int64_t t = 0; t < 2 * n_tiles; ++t) ranges[t] = 0;
    for (int64_t i = 0; i < m; ++i) {
        int64_t t = (int64_t)(keys[i] >> 32);
        if (i == 0 || (int64_t)(keys[i - 1] >> 32) != t) ranges[2 * t] = (int32_t)i;
        if (i == m - 1 || (int64_t)(keys[i + 1] >> 32) != t) ranges[2 * t + 1] = (int32_t)(i + 1);
    }
}

/* ------------------------------------------------------------------------ */
/* Compositing (Sec. 2 Shader; Algorithm 1; Listing 1 evaluate).             */
/* For a pixel at raw coordinate (px, py), walk the ordered list:            */
/*   power = -(c00 dx^2 + 2 c01 dx dy + c11 dy^2)/2, d = px - mu_2D;         */
/*   skip if power > 0 (valid flag);                                         */
/*   alpha = min(alpha_max, o exp(power)); skip if alpha < alpha_t;          */
/*   stop (without accumulating) if T (1 - alpha) < T_eps;                   */
/*   C += c alpha T; T *= (1 - alpha).                                       */
/* Finally C += T bg.                                                        */
/*                                                                           */
/* Ambiguity band.  A float32 evaluation of the same walk may take a gate    */
/* decision the other way when the decision's margin is below the float32    */
/* uncertainty of the quantity compared.  bandm (NULL = no band) models that */
/* uncertainty per decision, as an absolute uncertainty of ln(alpha):        */
/*   u = eps (S + 1) + mu_abs m_i (|g_x| + |g_y|) + conic_rel Q_i,           */
/*   S = (|c00| dx^2 + 2 |c01 dx dy| + |c11| dy^2) / 2,  g = conic d,        */
/*   Q_i = (sa g_x^2 + 2 sb |g_x g_y| + sc g_y^2) / 2 + k_i |power|,         */
/* eps = relative precision of the float32 evaluation of the walk           */
/* (products, sums, the exponential).  The other two terms cover a float32  */
/* projection that computed its own records, with the per-primitive scales  */
/* unc[5 i ..] = (m_i, k_i, sa, sb, sc) of oracle_project_unc: m_i the      */
/* centre's rounding in pixels, Q_i the first-order effect of a relative    */
/* rounding of the Sigma_2D entries (g^T dSigma g / 2) plus the 2x2         */
/* inverse's cancellation k_i (NULL: m_i = 1, Q_i = S).  Both multipliers   */
/* are zero when both sides read the same float32 records.                  */
/* The relative uncertainty of T gathers                                     */
/* alpha_i u_i / (1 - alpha_i) + eps per blended entry, and the full factor  */
/* alpha / (1 - alpha) of an entry whose gate is ambiguous (its flip changes */
/* every later T by that factor).  A pixel is in the band (bit 1) when the   */
/* valid, alpha_t or T_eps decision lies within its uncertainty; bit 2 marks */
/* an ambiguous alpha_max clamp, which moves no value (min is continuous)    */
/* but switches a gradient.  jump (may be NULL) bounds how far the colour    */
/* can move through the flagged decisions: a flipped valid or alpha_t gate   */
/* moves it by at most alpha T (|c_i| + cmax) <= 2 cmax max(alpha, alpha_t) T*/
/* (the entry's own term and the rescaling of everything behind it), a       */
/* flipped stop by at most T cmax (the entry and everything behind it);      */
/* cmax bounds every colour and background channel.                          */
/* ------------------------------------------------------------------------ */

typedef struct {
    double eps, mu_abs, conic_rel, cmax;
} bandm;

static bandm read_band(const double *b) {
    bandm m = {0.0, 0.0, 0.0, 1.0};
    if (b) {
        m.eps = b[0];
        m.mu_abs = b[1];
        m.conic_rel = b[2];
        m.cmax = b[3];
    }
    return m;
}

typedef struct {
    int64_t idx;   /* primitive */
    int pos;       /* position in the walked list */
    double alpha, G, T; /* alpha, exp(power), transmittance before */
    int clamped;
    double dx, dy;
} contrib_t;

static int walk(double px, double py, const double *rec, const int64_t *list, int len, const ocfg *cfg,
                const bandm *bm, const double *unc, double C[3], double *Tout, int *last, int *band, double *jump,
                contrib_t *out, uint64_t *sig) {
    double T = 1.0, eT = 0.0, J = 0.0;
    C[0] = C[1] = C[2] = 0.0;
    int nc = 0, bd = 0;
    *last = 0;
    uint64_t h = sig ? *sig : 0;
    const double lat = log(cfg->at), lamax = log(cfg->amax), lteps = log(cfg->teps);
    for (int k = 0; k < len; ++k) {
        const double *R = rec + 12 * list[k];
        double dx = px - R[0], dy = py - R[1];
        double power = -0.5 * (R[2] * dx * dx + 2.0 * R[3] * dx * dy + R[4] * dy * dy);
        double u = 0.0;
        if (bm) {
            double S = 0.5 * (fabs(R[2]) * dx * dx + 2.0 * fabs(R[3] * dx * dy) + fabs(R[4]) * dy * dy);
            double gx = R[2] * dx + R[3] * dy, gy = R[3] * dx + R[4] * dy;
            double mi = 1.0, cs = S;
            if (unc) {
                const double *U = unc + 5 * list[k];
                mi = U[0];
                cs = 0.5 * (U[2] * gx * gx + 2.0 * U[3] * fabs(gx * gy) + U[4] * gy * gy) + U[1] * fabs(power);
            }
            u = bm->eps * (S + 1.0) + bm->mu_abs * mi * (fabs(gx) + fabs(gy)) + bm->conic_rel * cs;
            double am = R[5] < cfg->amax ? R[5] : cfg->amax;
            if (power > -u) { /* valid gate ambiguous (pixel at the centre) */
                bd |= 1;
                J += 2.0 * bm->cmax * am * T;
                eT += am / (1.0 - am);
            }
        }
        if (power > 0.0) continue;
        double G = exp(power);
        double og = R[5] * G;
        double alpha = og < cfg->amax ? og : cfg->amax;
        if (bm) {
            double la = log(R[5]) + power;
            if (fabs(la - lamax) <= u) bd |= 2;
            if (fabs(la - lat) <= u) {
                double am = alpha > cfg->at ? alpha : cfg->at;
                bd |= 1;
                J += 2.0 * bm->cmax * am * T;
                eT += am / (1.0 - am);
            }
        }
        if (alpha < cfg->at) continue;
        double tt = T * (1.0 - alpha);
        if (bm) {
            double ut = eT + alpha * u / (1.0 - alpha) + bm->eps;
            if (fabs(log(tt) - lteps) <= ut) {
                bd |= 1;
                J += bm->cmax * T;
            }
        }
        if (tt < cfg->teps) {
            h = h * 1099511628211ULL ^ 0xffffULL;
            break;
        }
        if (out) {
            out[nc].idx = list[k];
            out[nc].pos = k;
            out[nc].alpha = alpha;
            out[nc].G = G;
            out[nc].T = T;
            out[nc].clamped = !(og < cfg->amax);
            out[nc].dx = dx;
            out[nc].dy = dy;
        }
        h = (h ^ (uint64_t)(list[k] + 1)) * 1099511628211ULL;
        for (int c = 0; c < 3; ++c) C[c] += R[6 + c] * alpha * T;
        T = tt;
        if (bm) eT += alpha * u / (1.0 - alpha) + bm->eps;
        ++nc;
        *last = k + 1;
    }
    for (int c = 0; c < 3; ++c) C[c] += T * cfg->bg[c];
    *Tout = T;
    *band = bd;
    if (jump) *jump = J;
    if (sig) *sig = h;
    return nc;
}

typedef struct {
    uint32_t key;
    int64_t idx;
} dz_t;

static int dz_cmp(const void *a, const void *b) {
    const dz_t *x = (const dz_t *)a, *y = (const dz_t *)b;
    if (x->key != y->key) return x->key < y->key ? -1 : 1;
    return x->idx < y->idx ? -1 : (x->idx > y->idx ? 1 : 0);
}

/* Visible primitives ordered by (float32 bits of the depth key, index): the order of the sorted
 * tile lists within every tile.  key[n] from oracle_depth_keys; NULL = the record's FP64 depth
 * rounded to float32 (equal to the key when the view matrix is the identity).  Depths of visible
 * primitives are positive, so the bit order is the value order. */
static int64_t depth_order(int64_t n, const double *rec, const float *key, int64_t *order) {
    dz_t *a = (dz_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(dz_t));
    int64_t m = 0;
    for (int64_t i = 0; i < n; ++i)
        if (rec[12 * i + 11] != 0.0) {
            a[m].key = f32_bits(key ? key[i] : (float)rec[12 * i + 9]);
            a[m].idx = i;
            ++m;
        }
    qsort(a, (size_t)m, sizeof(dz_t), dz_cmp);
    for (int64_t i = 0; i < m; ++i) order[i] = a[i].idx;
    free(a);
    return m;
}

/* Brute force (no tiles): every visible primitive at every listed pixel, in depth-key order.
 * pix[npix*2] = (x, y) integer pixel coordinates; out color[npix*3], tfinal[npix], band[npix],
 * jump[npix] (may be NULL); bandp[4] = (eps, mu_abs, conic_rel, cmax) or NULL; unc[n*5] per
 * primitive uncertainty scales (oracle_project_unc) or NULL; psig[npix] (may be NULL) = hash of
 * each pixel's decisions (blended entries and the stop), sig (may be NULL) = hash of them all. */
void oracle_render_pixels(int64_t n, const double *rec, const float *key, const int32_t *pix, int64_t npix,
                          const double *cfgv, const double *bandp, const double *unc, double *color, double *tfinal,
                          int32_t *band, double *jump, uint64_t *psig, uint64_t *sig) {
    ocfg cfg = read_cfg(cfgv);
    bandm bm = read_band(bandp);
    int64_t *order = (int64_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int64_t));
    int64_t m = depth_order(n, rec, key, order);
    uint64_t hs = 1469598103934665603ULL;
    uint64_t *hp = (uint64_t *)malloc((size_t)(npix > 0 ? npix : 1) * sizeof(uint64_t));
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t p = 0; p < npix; ++p) {
        double C[3], T, J;
        int last, bd;
        uint64_t h = (uint64_t)p;
        walk((double)pix[2 * p], (double)pix[2 * p + 1], rec, order, (int)m, &cfg, bandp ? &bm : NULL, unc, C, &T,
             &last, &bd, &J, NULL, &h);
        for (int c = 0; c < 3; ++c) color[3 * p + c] = C[c];
        tfinal[p] = T;
        band[p] = bd;
        if (jump) jump[p] = J;
        if (psig) psig[p] = h;
        hp[p] = h;
    }
    for (int64_t p = 0; p < npix; ++p) hs = (hs ^ hp[p]) * 1099511628211ULL;
    if (sig) *sig = hs;
    free(hp);
    free(order);
}

/* Per-tile walk over given lists: vals[ranges[t,0]:ranges[t,1]] for tile t.
 * image[3,H,W] (planar), tfinal[H,W], ncontrib[H,W] (position+1 of the last
 * accumulated entry in the tile's list), band[H,W], jump[H,W] (may be NULL). */
void oracle_render_tiles(int64_t n, const double *rec, const uint32_t *vals, const int32_t *ranges,
                         const double *camv, const double *cfgv, const double *bandp, const double *unc,
                         double *image, double *tfinal, int32_t *ncontrib, int32_t *band, double *jump) {
    (void)n;
    ocam cam = read_cam(camv);
    ocfg cfg = read_cfg(cfgv);
    bandm bm = read_band(bandp);
    int Wt = (cam.W + cfg.tw - 1) / cfg.tw, Ht = (cam.H + cfg.th - 1) / cfg.th;
    int64_t HW = (int64_t)cam.W * cam.H;
#pragma omp parallel for schedule(dynamic, 1)
    for (int t = 0; t < Wt * Ht; ++t) {
        int tx = t % Wt, ty = t / Wt;
        int s = ranges[2 * t], e = ranges[2 * t + 1];
        int len = e - s;
        int64_t *list = (int64_t *)malloc((size_t)(len > 0 ? len : 1) * sizeof(int64_t));
        for (int k = 0; k < len; ++k) list[k] = vals[s + k];
        for (int yy = 0; yy < cfg.th; ++yy)
            for (int xx = 0; xx < cfg.tw; ++xx) {
                int x = tx * cfg.tw + xx, y = ty * cfg.th + yy;
                if (x >= cam.W || y >= cam.H) continue;
                double C[3], T, J;
                int last, bd;
                walk((double)x, (double)y, rec, list, len, &cfg, bandp ? &bm : NULL, unc, C, &T, &last, &bd, &J,
                     NULL, NULL);
                int64_t p = (int64_t)y * cam.W + x;
                for (int c = 0; c < 3; ++c) image[c * HW + p] = C[c];
                tfinal[p] = T;
                ncontrib[p] = last;
                band[p] = bd;
                if (jump) jump[p] = J;
            }
        free(list);
    }
}

/* ------------------------------------------------------------------------ */
/* Adjoint of compositing, written from the definition                       */
/*   C = sum_i c_i a_i T_i + T_N bg,  T_i = prod_{j<i} (1 - a_j):           */
/*   dC/dc_i = a_i T_i;                                                      */
/*   dC/da_i = c_i T_i - S_i / (1 - a_i),  S_i = sum_{j>i} c_j a_j T_j + T_N bg */
/* with S_i formed as an explicit suffix sum.  Through alpha = o exp(power)  */
/* (zero through the 0.99 clamp), power = -(c00 dx^2 + 2 c01 dx dy +         */
/* c11 dy^2)/2, dx = px - mx.  d_rec[n*12] accumulates (dmx, dmy, dc00,      */
/* dc01, dc11, do, dr, dg, db); entries 9..11 stay zero.                     */
/* ------------------------------------------------------------------------ */

static void pixel_adjoint(const double *rec, const contrib_t *cs, int nc, double Tfin, const double *g,
                          const ocfg *cfg, double *d_rec) {
    if (nc == 0) return;
    double *S = (double *)malloc((size_t)nc * 3 * sizeof(double));
    /* explicit suffix sums */
    for (int c = 0; c < 3; ++c) {
        double acc = Tfin * cfg->bg[c];
        for (int i = nc - 1; i >= 0; --i) {
            S[3 * i + c] = acc;
            acc += rec[12 * cs[i].idx + 6 + c] * cs[i].alpha * cs[i].T;
        }
    }
    for (int i = 0; i < nc; ++i) {
        const double *R = rec + 12 * cs[i].idx;
        double *D = d_rec + 12 * cs[i].idx;
        double a = cs[i].alpha, T = cs[i].T;
        double da = 0.0;
        for (int c = 0; c < 3; ++c) {
            D[6 + c] += g[c] * a * T;
            da += g[c] * (R[6 + c] * T - S[3 * i + c] / (1.0 - a));
        }
        if (cs[i].clamped) continue;
        /* alpha = o G, G = exp(power) */
        D[5] += da * cs[i].G;
        double dp = da * a; /* dL/dpower */
        double dx = cs[i].dx, dy = cs[i].dy;
        /* dpower/dc00 = -dx^2/2, dpower/dc01 = -dx dy, dpower/dc11 = -dy^2/2 */
        D[2] += dp * (-0.5 * dx * dx);
        D[3] += dp * (-dx * dy);
        D[4] += dp * (-0.5 * dy * dy);
        /* dpower/dmx = c00 dx + c01 dy ; dpower/dmy = c01 dx + c11 dy */
        D[0] += dp * (R[2] * dx + R[3] * dy);
        D[1] += dp * (R[3] * dx + R[4] * dy);
    }
    free(S);
}

/* Brute-force adjoint over all pixels of a W x H image (tiny scenes). */
void oracle_render_bwd_brute(int64_t n, const double *rec, const float *key, const double *camv, const double *cfgv,
                             const double *d_image, double *d_rec) {
    ocam cam = read_cam(camv);
    ocfg cfg = read_cfg(cfgv);
    int64_t *order = (int64_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int64_t));
    int64_t m = depth_order(n, rec, key, order);
    contrib_t *cs = (contrib_t *)malloc((size_t)(m > 0 ? m : 1) * sizeof(contrib_t));
    int64_t HW = (int64_t)cam.W * cam.H;
    memset(d_rec, 0, (size_t)n * 12 * sizeof(double));
    for (int y = 0; y < cam.H; ++y)
        for (int x = 0; x < cam.W; ++x) {
            int64_t p = (int64_t)y * cam.W + x;
            double g[3] = {d_image[p], d_image[HW + p], d_image[2 * HW + p]};
            if (g[0] == 0.0 && g[1] == 0.0 && g[2] == 0.0) continue;
            double C[3], T;
            int last, bd;
            int nc = walk((double)x, (double)y, rec, order, (int)m, &cfg, NULL, NULL, C, &T, &last, &bd, NULL, cs, NULL);
            pixel_adjoint(rec, cs, nc, T, g, &cfg, d_rec);
        }
    free(cs);
    free(order);
}

/* Per-tile adjoint over given lists (serial; deterministic). */
void oracle_render_bwd_tiles(int64_t n, const double *rec, const uint32_t *vals, const int32_t *ranges,
                             const double *camv, const double *cfgv, const double *d_image, double *d_rec) {
    ocam cam = read_cam(camv);
    ocfg cfg = read_cfg(cfgv);
    int Wt = (cam.W + cfg.tw - 1) / cfg.tw, Ht = (cam.H + cfg.th - 1) / cfg.th;
    int64_t HW = (int64_t)cam.W * cam.H;
    memset(d_rec, 0, (size_t)n * 12 * sizeof(double));
    for (int t = 0; t < Wt * Ht; ++t) {
        int tx = t % Wt, ty = t / Wt;
        int s = ranges[2 * t], e = ranges[2 * t + 1];
        int len = e - s;
        if (len <= 0) continue;
        int64_t *list = (int64_t *)malloc((size_t)len * sizeof(int64_t));
        contrib_t *cs = (contrib_t *)malloc((size_t)len * sizeof(contrib_t));
        for (int k = 0; k < len; ++k) list[k] = vals[s + k];
        for (int yy = 0; yy < cfg.th; ++yy)
            for (int xx = 0; xx < cfg.tw; ++xx) {
                int x = tx * cfg.tw + xx, y = ty * cfg.th + yy;
                if (x >= cam.W || y >= cam.H) continue;
                int64_t p = (int64_t)y * cam.W + x;
                double g[3] = {d_image[p], d_image[HW + p], d_image[2 * HW + p]};
                if (g[0] == 0.0 && g[1] == 0.0 && g[2] == 0.0) continue;
                double C[3], T;
                int last, bd;
                int nc = walk((double)x, (double)y, rec, list, len, &cfg, NULL, NULL, C, &T, &last, &bd, NULL, cs, NULL);
                pixel_adjoint(rec, cs, nc, T, g, &cfg, d_rec);
            }
        free(cs);
        free(list);
    }
}

/* ------------------------------------------------------------------------ */
/* Rendered features (the "rendered feature" class of the design space, e.g. */
/* depth and semantics): channel c of a pixel is sum_i f_ic alpha_i T_i over */
/* the same contributors and weights as the colour, with zero background.    */
/* feat[n*nfeat] are per-primitive feature rows; with_depth appends one      */
/* channel whose per-primitive value is the record's depth (camera z).       */
/* ------------------------------------------------------------------------ */

static double feat_value(const double *rec, const double *feat, int nfeat, int64_t i, int c) {
    return c < nfeat ? feat[(int64_t)nfeat * i + c] : rec[12 * i + 9];
}

void oracle_render_tiles_feat(int64_t n, const double *rec, const double *feat, int nfeat, int with_depth,
                              const uint32_t *vals, const int32_t *ranges, const double *camv, const double *cfgv,
                              double *image, double *features, double *tfinal) {
    ocam cam = read_cam(camv);
    ocfg cfg = read_cfg(cfgv);
    int Wt = (cam.W + cfg.tw - 1) / cfg.tw, Ht = (cam.H + cfg.th - 1) / cfg.th;
    int64_t HW = (int64_t)cam.W * cam.H;
    int nf = nfeat + (with_depth ? 1 : 0);
    (void)n;
#pragma omp parallel for schedule(dynamic, 1)
    for (int t = 0; t < Wt * Ht; ++t) {
        int tx = t % Wt, ty = t / Wt;
        int s0 = ranges[2 * t], e0 = ranges[2 * t + 1];
        int len = e0 - s0;
        int64_t *list = (int64_t *)malloc((size_t)(len > 0 ? len : 1) * sizeof(int64_t));
        contrib_t *cs = (contrib_t *)malloc((size_t)(len > 0 ? len : 1) * sizeof(contrib_t));
        for (int k = 0; k < len; ++k) list[k] = vals[s0 + k];
        for (int yy = 0; yy < cfg.th; ++yy)
            for (int xx = 0; xx < cfg.tw; ++xx) {
                int x = tx * cfg.tw + xx, y = ty * cfg.th + yy;
                if (x >= cam.W || y >= cam.H) continue;
                double C[3], T;
                int last, bd;
                int nc = walk((double)x, (double)y, rec, list, len, &cfg, NULL, NULL, C, &T, &last, &bd, NULL, cs, NULL);
                int64_t p = (int64_t)y * cam.W + x;
                for (int c = 0; c < 3; ++c) image[c * HW + p] = C[c];
                tfinal[p] = T;
                for (int c = 0; c < nf; ++c) {
                    double acc = 0.0;
                    for (int k = 0; k < nc; ++k) acc += feat_value(rec, feat, nfeat, cs[k].idx, c) * cs[k].alpha * cs[k].T;
                    features[c * HW + p] = acc;
                }
            }
        free(cs);
        free(list);
    }
}

/* Adjoint with features: the compositing adjoint over all channels (3 colours with background, nf
 * features without), dC/dalpha_i = sum_ch g_ch (v_ich T_i - S_ich / (1 - alpha_i)) with explicit
 * suffix sums, then through alpha as pixel_adjoint; d_feat[n*nfeat] and, for the depth channel,
 * d_rec[9] accumulate g alpha_i T_i. */
void oracle_render_bwd_tiles_feat(int64_t n, const double *rec, const double *feat, int nfeat, int with_depth,
                                  const uint32_t *vals, const int32_t *ranges, const double *camv, const double *cfgv,
                                  const double *d_image, const double *d_features, double *d_rec, double *d_feat) {
    ocam cam = read_cam(camv);
    ocfg cfg = read_cfg(cfgv);
    int Wt = (cam.W + cfg.tw - 1) / cfg.tw, Ht = (cam.H + cfg.th - 1) / cfg.th;
    int64_t HW = (int64_t)cam.W * cam.H;
    int nf = nfeat + (with_depth ? 1 : 0);
    int nch = 3 + nf;
    memset(d_rec, 0, (size_t)n * 12 * sizeof(double));
    if (nfeat > 0) memset(d_feat, 0, (size_t)n * nfeat * sizeof(double));
    for (int t = 0; t < Wt * Ht; ++t) {
        int tx = t % Wt, ty = t / Wt;
        int s0 = ranges[2 * t], e0 = ranges[2 * t + 1];
        int len = e0 - s0;
        if (len <= 0) continue;
        int64_t *list = (int64_t *)malloc((size_t)len * sizeof(int64_t));
        contrib_t *cs = (contrib_t *)malloc((size_t)len * sizeof(contrib_t));
        double *S = (double *)malloc((size_t)len * nch * sizeof(double));
        double *v = (double *)malloc((size_t)len * nch * sizeof(double));
        double *g = (double *)malloc((size_t)nch * sizeof(double));
        for (int k = 0; k < len; ++k) list[k] = vals[s0 + k];
        for (int yy = 0; yy < cfg.th; ++yy)
            for (int xx = 0; xx < cfg.tw; ++xx) {
                int x = tx * cfg.tw + xx, y = ty * cfg.th + yy;
                if (x >= cam.W || y >= cam.H) continue;
                int64_t p = (int64_t)y * cam.W + x;
                int any = 0;
                for (int c = 0; c < 3; ++c) any |= (g[c] = d_image[c * HW + p]) != 0.0;
                for (int c = 0; c < nf; ++c) any |= (g[3 + c] = d_features[c * HW + p]) != 0.0;
                if (!any) continue;
                double C[3], T;
                int last, bd;
                int nc = walk((double)x, (double)y, rec, list, len, &cfg, NULL, NULL, C, &T, &last, &bd, NULL, cs, NULL);
                if (nc == 0) continue;
                for (int i = 0; i < nc; ++i) {
                    for (int c = 0; c < 3; ++c) v[nch * i + c] = rec[12 * cs[i].idx + 6 + c];
                    for (int c = 0; c < nf; ++c) v[nch * i + 3 + c] = feat_value(rec, feat, nfeat, cs[i].idx, c);
                }
                for (int c = 0; c < nch; ++c) {
                    double acc = c < 3 ? T * cfg.bg[c] : 0.0;
                    for (int i = nc - 1; i >= 0; --i) {
                        S[nch * i + c] = acc;
                        acc += v[nch * i + c] * cs[i].alpha * cs[i].T;
                    }
                }
                for (int i = 0; i < nc; ++i) {
                    const double *R = rec + 12 * cs[i].idx;
                    double *D = d_rec + 12 * cs[i].idx;
                    double a = cs[i].alpha, Ti = cs[i].T;
                    double da = 0.0;
                    for (int c = 0; c < nch; ++c) da += g[c] * (v[nch * i + c] * Ti - S[nch * i + c] / (1.0 - a));
                    for (int c = 0; c < 3; ++c) D[6 + c] += g[c] * a * Ti;
                    for (int c = 0; c < nf; ++c) {
                        double gv = g[3 + c] * a * Ti;
                        if (c < nfeat) d_feat[(int64_t)nfeat * cs[i].idx + c] += gv;
                        else D[9] += gv;
                    }
                    if (cs[i].clamped) continue;
                    D[5] += da * cs[i].G;
                    double dp = da * a, dx = cs[i].dx, dy = cs[i].dy;
                    D[2] += dp * (-0.5 * dx * dx);
                    D[3] += dp * (-dx * dy);
                    D[4] += dp * (-0.5 * dy * dy);
                    D[0] += dp * (R[2] * dx + R[3] * dy);
                    D[1] += dp * (R[3] * dx + R[4] * dy);
                }
            }
        free(g);
        free(v);
        free(S);
        free(cs);
        free(list);
    }
}

/* ------------------------------------------------------------------------ */
/* Adjoint of the projection (Listing 1 project), from screen-space          */
/* gradients d_rec (dmx, dmy, dc00, dc01, dc11, do, dr, dg, db) to           */
/* dmu[n*3], dscale[n*3], dquat[n*4], dopac[n], dsh[n*K*3].                  */
/* Chain: conic = Sigma_2D^{-1} (d(A^{-1}) = -A^{-1} dA A^{-1});             */
/* Sigma_2D = T Sigma T^T + dil I, T = J W; J(camera point) with the clamp;   */
/* camera point = W mu + t; Sigma = M M^T, M = R(q/|q|) diag(s);             */
/* mu_2D = (fx x/z + cx, fy y/z + cy); rgb = max(0, sum sh Y(d) + 0.5),      */
/* d = (mu - campos)/|mu - campos|.  Invisible primitives get zero.          */
/* ------------------------------------------------------------------------ */

/* d R / d qn_k for the unit-quaternion rotation (w, x, y, z) */
static void drot_dq(const double *qn, double dR[4][9]) {
    double w = qn[0], x = qn[1], y = qn[2], z = qn[3];
    /* w */
    double Dw[9] = {0, -2 * z, 2 * y, 2 * z, 0, -2 * x, -2 * y, 2 * x, 0};
    /* x */
    double Dx[9] = {0, 2 * y, 2 * z, 2 * y, -4 * x, -2 * w, 2 * z, 2 * w, -4 * x};
    /* y */
    double Dy[9] = {-4 * y, 2 * x, 2 * w, 2 * x, 0, 2 * z, -2 * w, 2 * z, -4 * y};
    /* z */
    double Dz[9] = {-4 * z, -2 * w, 2 * x, 2 * w, -4 * z, 2 * y, 2 * x, 2 * y, 0};
    memcpy(dR[0], Dw, sizeof(Dw));
    memcpy(dR[1], Dx, sizeof(Dx));
    memcpy(dR[2], Dy, sizeof(Dy));
    memcpy(dR[3], Dz, sizeof(Dz));
}

void oracle_project_bwd(int64_t n, const double *mu, const double *scale, const double *quat, const double *opac,
                        const double *sh, const double *camv, const double *cfgv, const double *d_rec,
                        double *dmu, double *dscale, double *dquat, double *dopac, double *dsh) {
    ocam cam = read_cam(camv);
    ocfg cfg = read_cfg(cfgv);
    int K = (cfg.deg + 1) * (cfg.deg + 1);
    const double *V = cam.V;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        oproj P;
        const double *D = d_rec + 12 * i;
        const double *s = scale + 3 * i;
        const double *shi = sh + (int64_t)3 * K * i;
        double *gmu = dmu + 3 * i, *gs = dscale + 3 * i, *gq = dquat + 4 * i, *gsh = dsh + (int64_t)3 * K * i;
        project_one(mu + 3 * i, s, quat + 4 * i, opac[i], shi, &cam, &cfg, &P);
        memset(gmu, 0, 3 * sizeof(double));
        memset(gs, 0, 3 * sizeof(double));
        memset(gq, 0, 4 * sizeof(double));
        memset(gsh, 0, (size_t)3 * K * sizeof(double));
        dopac[i] = 0.0;
        if (!P.visible) continue;
        dopac[i] = D[5];

        /* colour */
        double Y[16], dY[48];
        oracle_sh_basis(cfg.deg, P.dir, Y, dY);
        double gdir[3] = {0, 0, 0};
        for (int c = 0; c < 3; ++c) {
            if (!(P.raw[c] > 0.0)) continue;
            double g = D[6 + c];
            for (int k = 0; k < K; ++k) {
                gsh[3 * k + c] = Y[k] * g;
                for (int j = 0; j < 3; ++j) gdir[j] += g * shi[3 * k + c] * dY[3 * k + j];
            }
        }
        double dd = gdir[0] * P.dir[0] + gdir[1] * P.dir[1] + gdir[2] * P.dir[2];
        for (int j = 0; j < 3; ++j) gmu[j] += (gdir[j] - P.dir[j] * dd) / P.vlen;

        /* camera-space point gradient */
        double x = P.mc[0], y = P.mc[1], z = P.mc[2];
        double gmc[3] = {0, 0, 0};
        gmc[0] += D[0] * cam.fx / z;
        gmc[1] += D[1] * cam.fy / z;
        gmc[2] += -D[0] * cam.fx * x / (z * z) - D[1] * cam.fy * y / (z * z);

        /* conic -> Sigma_2D : dL/dA = -A^{-1} G A^{-1}, G symmetric with the
         * off-diagonal record entry split over both matrix entries */
        double Ai[4] = {P.conic[0], P.conic[1], P.conic[1], P.conic[2]};
        double G[4] = {D[2], 0.5 * D[3], 0.5 * D[3], D[4]};
        double AG[4], GA[4];
        for (int r = 0; r < 2; ++r)
            for (int c = 0; c < 2; ++c) {
                AG[2 * r + c] = Ai[2 * r] * G[c] + Ai[2 * r + 1] * G[2 + c];
            }
        for (int r = 0; r < 2; ++r)
            for (int c = 0; c < 2; ++c) GA[2 * r + c] = -(AG[2 * r] * Ai[c] + AG[2 * r + 1] * Ai[2 + c]);
        /* GA = dL/dSigma_2D as a symmetric matrix (equal to dL/d(T Sigma T^T)) */

        /* Sigma_2D' = T Sigma T^T : dL/dSigma = T^T GA T ; dL/dT = 2 GA T Sigma */
        double gSig[9];
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) {
                double acc = 0.0;
                for (int r = 0; r < 2; ++r)
                    for (int c = 0; c < 2; ++c) acc += P.Tm[3 * r + a] * GA[2 * r + c] * P.Tm[3 * c + b];
                gSig[3 * a + b] = acc;
            }
        double gT[6];
        for (int r = 0; r < 2; ++r)
            for (int b = 0; b < 3; ++b) {
                double acc = 0.0;
                for (int c = 0; c < 2; ++c)
                    for (int k = 0; k < 3; ++k) acc += GA[2 * r + c] * P.Tm[3 * c + k] * P.Sig[3 * k + b];
                gT[3 * r + b] = 2.0 * acc;
            }
        /* T = J W : dL/dJ = dL/dT W^T */
        double gJ[6];
        for (int r = 0; r < 2; ++r)
            for (int k = 0; k < 3; ++k) {
                double acc = 0.0;
                for (int b = 0; b < 3; ++b) acc += gT[3 * r + b] * V[4 * k + b];
                gJ[3 * r + k] = acc;
            }
        /* J00 = fx/z, J02 = -fx ux/z (ux = x/z unless clamped), J11, J12 alike */
        gmc[2] += gJ[0] * (-cam.fx / (z * z));
        gmc[2] += gJ[4] * (-cam.fy / (z * z));
        if (!P.clx) {
            /* J02 = -fx x / z^2 */
            gmc[0] += gJ[2] * (-cam.fx / (z * z));
            gmc[2] += gJ[2] * (2.0 * cam.fx * x / (z * z * z));
        } else {
            /* J02 = -fx L / z with L constant */
            gmc[2] += gJ[2] * (cam.fx * P.ux / (z * z));
        }
        if (!P.cly) {
            gmc[1] += gJ[5] * (-cam.fy / (z * z));
            gmc[2] += gJ[5] * (2.0 * cam.fy * y / (z * z * z));
        } else {
            gmc[2] += gJ[5] * (cam.fy * P.uy / (z * z));
        }
        /* rendered depth (record entry 9 = camera z) */
        gmc[2] += D[9];
        /* camera point = W mu + t */
        for (int j = 0; j < 3; ++j) gmu[j] += V[j] * gmc[0] + V[4 + j] * gmc[1] + V[8 + j] * gmc[2];

        /* Sigma = M M^T, M = R diag(s) : dL/dM = 2 gSig M (gSig symmetric) */
        double gSs[9];
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) gSs[3 * a + b] = 0.5 * (gSig[3 * a + b] + gSig[3 * b + a]);
        double gM[9];
        for (int a = 0; a < 3; ++a)
            for (int k = 0; k < 3; ++k) {
                double acc = 0.0;
                for (int b = 0; b < 3; ++b) acc += gSs[3 * a + b] * P.R[3 * b + k] * s[k];
                gM[3 * a + k] = 2.0 * acc;
            }
        double gR[9];
        for (int a = 0; a < 3; ++a)
            for (int k = 0; k < 3; ++k) {
                gs[k] += gM[3 * a + k] * P.R[3 * a + k];
                gR[3 * a + k] = gM[3 * a + k] * s[k];
            }
        double dR[4][9];
        drot_dq(P.qn, dR);
        double gqn[4];
        for (int j = 0; j < 4; ++j) {
            double acc = 0.0;
            for (int e = 0; e < 9; ++e) acc += gR[e] * dR[j][e];
            gqn[j] = acc;
        }
        /* qn = q / |q| */
        double dotq = gqn[0] * P.qn[0] + gqn[1] * P.qn[1] + gqn[2] * P.qn[2] + gqn[3] * P.qn[3];
        for (int j = 0; j < 4; ++j) gq[j] = (gqn[j] - P.qn[j] * dotq) / P.qnorm;
    }
}

/* ------------------------------------------------------------------------ */
/* 3DGUT (Appendix "Implementation of XPR-3DGUT"; Listing 3DGUT).           */
/* Projection by the unscented transform: 2n+1 = 7 sigma points of the 3D    */
/* Gaussian, X_0 = mu, X_{+-k} = mu +- sqrt(n + lambda) L_k with L = R S    */
/* (Sigma = L L^T), lambda = alpha^2 (n + kappa) - n, alpha = 1, beta = 2,  */
/* kappa = 0 (lambda = 0); weights w^m_0 = lambda/(n+lambda) = 0,         */
/* w^c_0 = w^m_0 + 1 - alpha^2 + beta = 2, w_i = 1/(2(n+lambda)) = 1/6.    */
/* Each point goes through the pinhole projection; mu_2D = sum w^m_i p_i,    */
/* Sigma_2D = sum w^c_i (p_i - mu_2D)(p_i - mu_2D)^T, then the low-pass      */
/* dilation (+ d I) with the Mip-Splatting opacity o' = o sqrt(det_0/det).   */
/* Pixel centres are at +0.5: the box uses mu_2D - 0.5, the cull extends the */
/* tiles' max bounds by one (tile_bounds).  Shader data: the camera centre   */
/* in the Gaussian's canonical frame, ro_c = M (c - mu), M = S^-1 R^T.       */
/* Evaluation along the pixel ray r(tau) = c + tau d (Eq. for tau_max):     */
/* d_c = M d, tau_max = -ro_c.d_c / d_c.d_c, and the largest response is     */
/* G = exp(-|ro_c + tau_max d_c|^2 / 2) = exp(-(|ro_c|^2 - (ro_c.d_c)^2 /   */
/* d_c.d_c)/2); valid iff G > 0.0113; alpha = min(alpha_max, o' G).         */
/* Record: the 12-float layout of 3DGS with the UT mean and conic, o', and   */
/* ln(o'/alpha_t); shader data sd[16] = ro_c[3], M[9] (row-major), o', rgb. */
/* ------------------------------------------------------------------------ */

/* Fisheye camera (equidistant projection with a radial polynomial; the model of the 3DGUT
 * configuration of this workload, not printed in the paper): a camera-space point (x, y, z) at angle
 * theta = atan2(r, z) from the axis, r = sqrt(x^2 + y^2), lands at
 *   u = fx theta_d x / r + cx,  v = fy theta_d y / r + cy,
 *   theta_d = theta (1 + k1 theta^2 + k2 theta^4 + k3 theta^6 + k4 theta^8)
 * (u = cx, v = cy on the axis).  The pixel ray inverts theta_d(theta) by Newton's method. */
static double fish_thetad(const ocam *cam, double th) {
    double t2 = th * th;
    return th * (1.0 + t2 * (cam->k[0] + t2 * (cam->k[1] + t2 * (cam->k[2] + t2 * cam->k[3]))));
}

static void fish_project(const ocam *cam, const double *pc, double *uv) {
    double r = sqrt(pc[0] * pc[0] + pc[1] * pc[1]);
    if (r == 0.0) {
        uv[0] = cam->cx;
        uv[1] = cam->cy;
        return;
    }
    double th = atan2(r, pc[2]);
    double s = fish_thetad(cam, th) / r;
    uv[0] = cam->fx * s * pc[0] + cam->cx;
    uv[1] = cam->fy * s * pc[1] + cam->cy;
}

void oracle_fisheye_project(const double *pc, const double *camv, double *uv) {
    ocam cam = read_cam(camv);
    fish_project(&cam, pc, uv);
}

/* d(u, v)/d(x, y, z) of the projection (pinhole or fisheye) as a 2x3 row-major matrix.  Fisheye,
 * with s = theta_d / r, t = theta_d'(theta) / (r^2 + z^2), K = (t z - s) / r^2:
 *   du/dx = fx (s + x^2 K), du/dy = fx x y K, du/dz = -fx x t, and v alike (K -> 2 (k1 - 1/3) / z^3
 *   and s -> 1 / z on the axis). */
static void proj_jacobian(const ocam *cam, const double *pc, double *J) {
    double x = pc[0], y = pc[1], z = pc[2];
    if (cam->model != 1) {
        J[0] = cam->fx / z;
        J[1] = 0.0;
        J[2] = -cam->fx * x / (z * z);
        J[3] = 0.0;
        J[4] = cam->fy / z;
        J[5] = -cam->fy * y / (z * z);
        return;
    }
    double r2 = x * x + y * y, r = sqrt(r2), s, t, K;
    if (r < 1e-9 * fabs(z)) {
        s = 1.0 / z;
        t = 1.0 / (z * z);
        K = 2.0 * (cam->k[0] - 1.0 / 3.0) / (z * z * z);
    } else {
        double th = atan2(r, z), t2 = th * th;
        double td = fish_thetad(cam, th);
        double tdp = 1.0 + t2 * (3.0 * cam->k[0] + t2 * (5.0 * cam->k[1] + t2 * (7.0 * cam->k[2] + t2 * 9.0 * cam->k[3])));
        s = td / r;
        t = tdp / (r2 + z * z);
        K = (t * z - s) / r2;
    }
    J[0] = cam->fx * (s + x * x * K);
    J[1] = cam->fx * x * y * K;
    J[2] = -cam->fx * x * t;
    J[3] = cam->fy * x * y * K;
    J[4] = cam->fy * (s + y * y * K);
    J[5] = -cam->fy * y * t;
}

/* camera-space unit direction of the fisheye pixel ray through image point (X, Y) */
static void fish_unproject(const ocam *cam, double X, double Y, double *dc) {
    double mx = (X - cam->cx) / cam->fx, my = (Y - cam->cy) / cam->fy;
    double td = sqrt(mx * mx + my * my);
    if (td == 0.0) {
        dc[0] = 0.0;
        dc[1] = 0.0;
        dc[2] = 1.0;
        return;
    }
    double th = td;
    for (int it = 0; it < 50; ++it) {
        double t2 = th * th;
        double f = fish_thetad(cam, th) - td;
        double fp = 1.0 + t2 * (3.0 * cam->k[0] + t2 * (5.0 * cam->k[1] + t2 * (7.0 * cam->k[2] + t2 * 9.0 * cam->k[3])));
        double step = f / fp;
        th -= step;
        if (fabs(step) <= 1e-15 * (1.0 + fabs(th))) break;
    }
    double st = sin(th);
    dc[0] = st * mx / td;
    dc[1] = st * my / td;
    dc[2] = cos(th);
}

#define UT_VALID 0.0113

typedef struct {
    double mu2d[2], cov0[3], cov[3], conic[3], det0, det, o, ln_thr, ex, ey, pre[4], mc[3], rgb[3], roc[3], M[9];
    double pts[7][2], pc[7][3], R[9], qn[4], qnorm, cp[3], dir[3], vlen, raw[3], mip;
    int bbox[4];
    int tc, visible;
} oproj_ut;

static void project_ut_one(const double *mu, const double *s, const double *q, double o, const double *sh,
                           const ocam *cam, const ocfg *cfg, oproj_ut *P) {
    memset(P, 0, sizeof(*P));
    const double *V = cam->V;
    for (int i = 0; i < 3; ++i) P->mc[i] = V[4 * i] * mu[0] + V[4 * i + 1] * mu[1] + V[4 * i + 2] * mu[2] + V[4 * i + 3];
    double *qn = P->qn, *R = P->R, *cp = P->cp, *dir = P->dir;
    quat_rot(q, qn, &P->qnorm, R);
    for (int i = 0; i < 3; ++i) cp[i] = -(V[i] * V[3] + V[4 + i] * V[7] + V[8 + i] * V[11]);
    /* colour as in 3DGS */
    double v[3] = {mu[0] - cp[0], mu[1] - cp[1], mu[2] - cp[2]};
    double vl = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
    P->vlen = vl;
    for (int i = 0; i < 3; ++i) dir[i] = v[i] / vl;
    int K = (cfg->deg + 1) * (cfg->deg + 1);
    double Y[16];
    oracle_sh_basis(cfg->deg, dir, Y, NULL);
    for (int c = 0; c < 3; ++c) {
        double acc = 0.5;
        for (int k = 0; k < K; ++k) acc += sh[3 * k + c] * Y[k];
        P->raw[c] = acc;
        P->rgb[c] = acc > 0.0 ? acc : 0.0;
    }
    /* shader data */
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) P->M[3 * i + j] = R[3 * j + i] / s[i];
    for (int i = 0; i < 3; ++i)
        P->roc[i] = P->M[3 * i] * (cp[0] - mu[0]) + P->M[3 * i + 1] * (cp[1] - mu[1]) + P->M[3 * i + 2] * (cp[2] - mu[2]);
    if (!(P->mc[2] > cam->z_near)) return;
    /* sigma points through the projection */
    const double sq3 = sqrt(3.0);
    double(*pts)[2] = P->pts;
    for (int k = 0; k < 7; ++k) {
        double X[3];
        int a = (k - 1) / 2;
        double sgn = (k == 0) ? 0.0 : ((k % 2) ? 1.0 : -1.0);
        for (int i = 0; i < 3; ++i) X[i] = mu[i] + (k == 0 ? 0.0 : sgn * sq3 * s[a] * R[3 * i + a]);
        double *pc = P->pc[k];
        for (int i = 0; i < 3; ++i) pc[i] = V[4 * i] * X[0] + V[4 * i + 1] * X[1] + V[4 * i + 2] * X[2] + V[4 * i + 3];
        if (!(pc[2] > cam->z_near)) return; /* a sigma point behind the near plane: footprint undefined */
        if (cam->model == 1) {
            fish_project(cam, pc, pts[k]);
        } else {
            pts[k][0] = cam->fx * pc[0] / pc[2] + cam->cx;
            pts[k][1] = cam->fy * pc[1] / pc[2] + cam->cy;
        }
    }
    const double wm[7] = {0.0, 1.0 / 6, 1.0 / 6, 1.0 / 6, 1.0 / 6, 1.0 / 6, 1.0 / 6};
    const double wc[7] = {2.0, 1.0 / 6, 1.0 / 6, 1.0 / 6, 1.0 / 6, 1.0 / 6, 1.0 / 6};
    for (int k = 0; k < 7; ++k) {
        P->mu2d[0] += wm[k] * pts[k][0];
        P->mu2d[1] += wm[k] * pts[k][1];
    }
    for (int k = 0; k < 7; ++k) {
        double dx = pts[k][0] - P->mu2d[0], dy = pts[k][1] - P->mu2d[1];
        P->cov0[0] += wc[k] * dx * dx;
        P->cov0[1] += wc[k] * dx * dy;
        P->cov0[2] += wc[k] * dy * dy;
    }
    P->det0 = P->cov0[0] * P->cov0[2] - P->cov0[1] * P->cov0[1];
    P->cov[0] = P->cov0[0] + cfg->dil;
    P->cov[1] = P->cov0[1];
    P->cov[2] = P->cov0[2] + cfg->dil;
    P->det = P->cov[0] * P->cov[2] - P->cov[1] * P->cov[1];
    if (!(P->det > 0.0)) return;
    P->mip = sqrt((P->det0 > 0.0 ? P->det0 : 0.0) / P->det);
    P->o = o * P->mip;
    if (!(P->o > cfg->at)) return; /* strict for 3DGUT (its projection listing), unlike 3DGS */
    P->conic[0] = P->cov[2] / P->det;
    P->conic[1] = -P->cov[1] / P->det;
    P->conic[2] = P->cov[0] / P->det;
    P->ln_thr = log(P->o / cfg->at);
    P->ex = sqrt(2.0 * P->ln_thr * P->cov[0]);
    P->ey = sqrt(2.0 * P->ln_thr * P->cov[2]);
    double r = P->ex > P->ey ? P->ex : P->ey;
    int Wt = (cam->W + cfg->tw - 1) / cfg->tw, Ht = (cam->H + cfg->th - 1) / cfg->th;
    /* the box in pixel-index coordinates: mu_2D - 0.5 (ray offset) */
    P->pre[0] = (P->mu2d[0] - 0.5 - P->ex) / cfg->tw;
    P->pre[1] = (P->mu2d[1] - 0.5 - P->ey) / cfg->th;
    P->pre[2] = (P->mu2d[0] - 0.5 + P->ex) / cfg->tw;
    P->pre[3] = (P->mu2d[1] - 0.5 + P->ey) / cfg->th;
    P->bbox[0] = (int)clampd(floor(P->pre[0]), 0.0, (double)Wt);
    P->bbox[1] = (int)clampd(floor(P->pre[1]), 0.0, (double)Ht);
    P->bbox[2] = (int)clampd(floor(P->pre[2]) + 1.0, 0.0, (double)Wt);
    P->bbox[3] = (int)clampd(floor(P->pre[3]) + 1.0, 0.0, (double)Ht);
    int tc = (P->bbox[2] - P->bbox[0]) * (P->bbox[3] - P->bbox[1]);
    P->visible = (r > 0.0) && (tc > 0);
    P->tc = P->visible ? tc : 0;
    if (!P->visible) memset(P->bbox, 0, sizeof(P->bbox));
}

/* rec[n*12] (3DGS layout: UT mean, conic, o', rgb, depth, ln(o'/a_t), visible), sd[n*16],
 * bbox[n*4], tc[n]; pre[n*4] and cov0[n*3] (Sigma_2D before the dilation) may be NULL. */
void oracle_project_ut(int64_t n, const double *mu, const double *scale, const double *quat, const double *opac,
                       const double *sh, const double *camv, const double *cfgv, double *rec, double *sd,
                       int32_t *bbox, int32_t *tc, double *pre, double *cov0) {
    ocam cam = read_cam(camv);
    ocfg cfg = read_cfg(cfgv);
    int K = (cfg.deg + 1) * (cfg.deg + 1);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        oproj_ut P;
        project_ut_one(mu + 3 * i, scale + 3 * i, quat + 4 * i, opac[i], sh + (int64_t)3 * K * i, &cam, &cfg, &P);
        double *r = rec + 12 * i, *d = sd + 16 * i;
        memset(r, 0, 12 * sizeof(double));
        r[9] = P.mc[2];
        for (int j = 0; j < 3; ++j) d[j] = P.roc[j];
        for (int j = 0; j < 9; ++j) d[3 + j] = P.M[j];
        d[12] = P.visible ? P.o : 0.0;
        for (int j = 0; j < 3; ++j) d[13 + j] = P.visible ? P.rgb[j] : 0.0;
        if (P.visible) {
            r[0] = P.mu2d[0];
            r[1] = P.mu2d[1];
            r[2] = P.conic[0];
            r[3] = P.conic[1];
            r[4] = P.conic[2];
            r[5] = P.o;
            r[6] = P.rgb[0];
            r[7] = P.rgb[1];
            r[8] = P.rgb[2];
            r[10] = P.ln_thr;
            r[11] = 1.0;
        }
        for (int j = 0; j < 4; ++j) bbox[4 * i + j] = P.bbox[j];
        tc[i] = P.tc;
        if (pre)
            for (int j = 0; j < 4; ++j) pre[4 * i + j] = P.visible ? P.pre[j] : 0.0;
        if (cov0)
            for (int j = 0; j < 3; ++j) cov0[3 * i + j] = P.cov0[j];
    }
}

/* pixel_info: the world-space unit ray direction through the centre (x + 0.5, y + 0.5). */
static void pixel_ray(double x, double y, const ocam *cam, double *rd) {
    double dc[3] = {(x + 0.5 - cam->cx) / cam->fx, (y + 0.5 - cam->cy) / cam->fy, 1.0};
    if (cam->model == 1) {
        fish_unproject(cam, x + 0.5, y + 0.5, dc);
    } else {
        double nl = sqrt(dc[0] * dc[0] + dc[1] * dc[1] + dc[2] * dc[2]);
        for (int i = 0; i < 3; ++i) dc[i] /= nl;
    }
    const double *V = cam->V; /* R_c2w = R_w2c^T */
    for (int i = 0; i < 3; ++i) rd[i] = V[i] * dc[0] + V[4 + i] * dc[1] + V[8 + i] * dc[2];
}

/* largest response of the Gaussian of shader data S along the ray of direction rd; tau (the
 * maximiser tau_max in the canonical frame's parametrisation) and e = ro_c + tau d_c on request */
static double ut_response_full(const double *S, const double *rd, double *tau_out, double *e_out) {
    double dcn[3];
    for (int i = 0; i < 3; ++i) dcn[i] = S[3 + 3 * i] * rd[0] + S[4 + 3 * i] * rd[1] + S[5 + 3 * i] * rd[2];
    double a = S[0] * dcn[0] + S[1] * dcn[1] + S[2] * dcn[2];
    double b = dcn[0] * dcn[0] + dcn[1] * dcn[1] + dcn[2] * dcn[2];
    double tau = -a / b;
    double e[3] = {S[0] + tau * dcn[0], S[1] + tau * dcn[1], S[2] + tau * dcn[2]};
    if (tau_out) *tau_out = tau;
    if (e_out)
        for (int i = 0; i < 3; ++i) e_out[i] = e[i];
    return exp(-0.5 * (e[0] * e[0] + e[1] * e[1] + e[2] * e[2]));
}

static double ut_response(const double *S, const double *rd) { return ut_response_full(S, rd, NULL, NULL); }

double oracle_ut_response(const double *sd, const double *rd) { return ut_response(sd, rd); }

typedef struct {
    int64_t idx;
    double alpha, G, T, tau, e[3];
    int clamped;
} contrib_ut;

/* The walk of the 3DGS compositing with the ray response in place of the 2D one.  out (may be
 * NULL) records the contributors; sig (may be NULL) hashes every decision taken.  Band: a decision
 * is ambiguous when its quantity lies within a relative delta of its threshold (valid, alpha_t,
 * alpha_max) or, for the T_eps stop, within the relative uncertainty T has gathered (delta
 * alpha / (1 - alpha) per blended entry, the full alpha / (1 - alpha) of an ambiguous gate).  jump
 * (may be NULL) bounds the colour change through the flagged decisions in units of the largest
 * colour magnitude (2 max(alpha, alpha_t) T per flipped gate, T per flipped stop), as for 3DGS. */
static int walk_ut(const double *rd, const double *sd, const int64_t *list, int len, const ocfg *cfg, double delta,
                   double C[3], double *Tout, int *last, int *band, double *jump, contrib_ut *out, uint64_t *sig) {
    double T = 1.0, eT = 0.0, J = 0.0;
    C[0] = C[1] = C[2] = 0.0;
    int nc = 0, bd = 0;
    uint64_t h = sig ? *sig : 0;
    *last = 0;
    for (int k = 0; k < len; ++k) {
        const double *S = sd + 16 * list[k];
        double tau, e[3];
        double G = ut_response_full(S, rd, &tau, e);
        double og = S[12] * G;
        double alpha = og < cfg->amax ? og : cfg->amax;
        double am = alpha > cfg->at ? alpha : cfg->at;
        if (delta > 0.0 && (fabs(G - UT_VALID) <= delta * UT_VALID || fabs(alpha - cfg->at) <= delta * cfg->at)) {
            bd |= 1;
            J += 2.0 * am * T;
            eT += am / (1.0 - am);
        }
        if (!(G > UT_VALID)) continue;
        if (delta > 0.0 && fabs(og - cfg->amax) <= delta * cfg->amax) bd |= 2;
        if (alpha < cfg->at) continue;
        double tt = T * (1.0 - alpha);
        if (delta > 0.0 && fabs(log(tt / cfg->teps)) <= eT + alpha * delta / (1.0 - alpha) + delta) {
            bd |= 1;
            J += T;
        }
        if (tt < cfg->teps) {
            h = h * 1099511628211ULL ^ 0xffffULL;
            break;
        }
        if (out) {
            out[nc].idx = list[k];
            out[nc].alpha = alpha;
            out[nc].G = G;
            out[nc].T = T;
            out[nc].tau = tau;
            for (int i = 0; i < 3; ++i) out[nc].e[i] = e[i];
            out[nc].clamped = !(og < cfg->amax);
        }
        h = (h ^ (uint64_t)(list[k] + 1)) * 1099511628211ULL;
        for (int c = 0; c < 3; ++c) C[c] += S[13 + c] * alpha * T;
        T = tt;
        eT += alpha * delta / (1.0 - alpha) + delta;
        ++nc;
        *last = k + 1;
    }
    for (int c = 0; c < 3; ++c) C[c] += T * cfg->bg[c];
    *Tout = T;
    *band = bd;
    if (jump) *jump = J;
    if (sig) *sig = h;
    return nc;
}

/* Per-tile walk of 3DGUT over given lists (as oracle_render_tiles). */
void oracle_render_tiles_ut(int64_t n, const double *rec, const double *sd, const uint32_t *vals,
                            const int32_t *ranges, const double *camv, const double *cfgv, double delta,
                            double *image, double *tfinal, int32_t *ncontrib, int32_t *band, double *jump,
                            uint64_t *psig) {
    (void)n;
    ocam cam = read_cam(camv);
    ocfg cfg = read_cfg(cfgv);
    int Wt = (cam.W + cfg.tw - 1) / cfg.tw, Ht = (cam.H + cfg.th - 1) / cfg.th;
    int64_t HW = (int64_t)cam.W * cam.H;
#pragma omp parallel for schedule(dynamic, 1)
    for (int t = 0; t < Wt * Ht; ++t) {
        int tx = t % Wt, ty = t / Wt;
        int s0 = ranges[2 * t], e0 = ranges[2 * t + 1];
        int len = e0 - s0;
        int64_t *list = (int64_t *)malloc((size_t)(len > 0 ? len : 1) * sizeof(int64_t));
        for (int k = 0; k < len; ++k) list[k] = vals[s0 + k];
        for (int yy = 0; yy < cfg.th; ++yy)
            for (int xx = 0; xx < cfg.tw; ++xx) {
                int x = tx * cfg.tw + xx, y = ty * cfg.th + yy;
                if (x >= cam.W || y >= cam.H) continue;
                double rd[3], C[3], T, J;
                int last, bd;
                uint64_t h = 0;
                pixel_ray((double)x, (double)y, &cam, rd);
                walk_ut(rd, sd, list, len, &cfg, delta, C, &T, &last, &bd, &J, NULL, &h);
                int64_t p = (int64_t)y * cam.W + x;
                if (jump) jump[p] = J;
                if (psig) psig[p] = h;
                for (int c = 0; c < 3; ++c) image[c * HW + p] = C[c];
                tfinal[p] = T;
                ncontrib[p] = last;
                band[p] = bd;
            }
        free(list);
    }
}

/* 3DGUT without tiles: every visible primitive (depth order) at every listed pixel. */
void oracle_render_pixels_ut(int64_t n, const double *rec, const double *sd, const float *key, const int32_t *pix,
                             int64_t npix, const double *camv, const double *cfgv, double delta, double *color,
                             double *tfinal, int32_t *band, double *jump) {
    ocam cam = read_cam(camv);
    ocfg cfg = read_cfg(cfgv);
    int64_t *order = (int64_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int64_t));
    int64_t m = depth_order(n, rec, key, order);
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t p = 0; p < npix; ++p) {
        double rd[3], C[3], T, J;
        int last, bd;
        pixel_ray((double)pix[2 * p], (double)pix[2 * p + 1], &cam, rd);
        walk_ut(rd, sd, order, (int)m, &cfg, delta, C, &T, &last, &bd, &J, NULL, NULL);
        if (jump) jump[p] = J;
        for (int c = 0; c < 3; ++c) color[3 * p + c] = C[c];
        tfinal[p] = T;
        band[p] = bd;
    }
    free(order);
}

void oracle_pixel_ray(int x, int y, const double *camv, double *rd) {
    ocam cam = read_cam(camv);
    pixel_ray((double)x, (double)y, &cam, rd);
}

/* ------------------------------------------------------------------------ */
/* Adjoint of 3DGUT.  Compositing as in 3DGS (dC/dc_i, dC/da_i with explicit */
/* suffix sums), then through alpha = o' G (nothing through the clamp) and   */
/* G = exp(-Q/2), Q = |ro_c|^2 - (ro_c.d_c)^2 / (d_c.d_c), d_c = M d:        */
/*   dQ/dro_c = 2 e,  dQ/dd_c = 2 tau e,  e = ro_c + tau d_c,                */
/*   dL/dM_ij = dL/dd_c_i d_j.                                               */
/* d_sd[n*16] accumulates (dro_c[3], dM[9], do', drgb[3]).                   */
/* ------------------------------------------------------------------------ */

static void pixel_adjoint_ut(const double *sd, const contrib_ut *cs, int nc, double Tfin, const double *g,
                             const double *rd, const ocfg *cfg, double *d_sd) {
    if (nc == 0) return;
    double *S = (double *)malloc((size_t)nc * 3 * sizeof(double));
    for (int c = 0; c < 3; ++c) {
        double acc = Tfin * cfg->bg[c];
        for (int i = nc - 1; i >= 0; --i) {
            S[3 * i + c] = acc;
            acc += sd[16 * cs[i].idx + 13 + c] * cs[i].alpha * cs[i].T;
        }
    }
    for (int i = 0; i < nc; ++i) {
        const double *Sd = sd + 16 * cs[i].idx;
        double *D = d_sd + 16 * cs[i].idx;
        double a = cs[i].alpha, T = cs[i].T;
        double da = 0.0;
        for (int c = 0; c < 3; ++c) {
            D[13 + c] += g[c] * a * T;
            da += g[c] * (Sd[13 + c] * T - S[3 * i + c] / (1.0 - a));
        }
        if (cs[i].clamped) continue;
        D[12] += da * cs[i].G;
        double dQ = -0.5 * cs[i].G * (da * Sd[12]); /* dL/dQ = dL/dG dG/dQ */
        const double *e = cs[i].e;
        for (int r = 0; r < 3; ++r) {
            D[r] += 2.0 * dQ * e[r];
            double ddc = 2.0 * dQ * cs[i].tau * e[r];
            for (int j = 0; j < 3; ++j) D[3 + 3 * r + j] += ddc * rd[j];
        }
    }
    free(S);
}

/* Per-tile adjoint over given lists (serial; deterministic). */
void oracle_render_bwd_tiles_ut(int64_t n, const double *sd, const uint32_t *vals, const int32_t *ranges,
                                const double *camv, const double *cfgv, const double *d_image, double *d_sd) {
    ocam cam = read_cam(camv);
    ocfg cfg = read_cfg(cfgv);
    int Wt = (cam.W + cfg.tw - 1) / cfg.tw, Ht = (cam.H + cfg.th - 1) / cfg.th;
    int64_t HW = (int64_t)cam.W * cam.H;
    memset(d_sd, 0, (size_t)n * 16 * sizeof(double));
    for (int t = 0; t < Wt * Ht; ++t) {
        int tx = t % Wt, ty = t / Wt;
        int s0 = ranges[2 * t], e0 = ranges[2 * t + 1];
        int len = e0 - s0;
        if (len <= 0) continue;
        int64_t *list = (int64_t *)malloc((size_t)len * sizeof(int64_t));
        contrib_ut *cs = (contrib_ut *)malloc((size_t)len * sizeof(contrib_ut));
        for (int k = 0; k < len; ++k) list[k] = vals[s0 + k];
        for (int yy = 0; yy < cfg.th; ++yy)
            for (int xx = 0; xx < cfg.tw; ++xx) {
                int x = tx * cfg.tw + xx, y = ty * cfg.th + yy;
                if (x >= cam.W || y >= cam.H) continue;
                int64_t p = (int64_t)y * cam.W + x;
                double g[3] = {d_image[p], d_image[HW + p], d_image[2 * HW + p]};
                if (g[0] == 0.0 && g[1] == 0.0 && g[2] == 0.0) continue;
                double rd[3], C[3], T;
                int last, bd;
                pixel_ray((double)x, (double)y, &cam, rd);
                int nc = walk_ut(rd, sd, list, len, &cfg, 0.0, C, &T, &last, &bd, NULL, cs, NULL);
                pixel_adjoint_ut(sd, cs, nc, T, g, rd, &cfg, d_sd);
            }
        free(cs);
        free(list);
    }
}

/* Adjoint of the 3DGUT projection: d_sd (dro_c, dM, do', drgb) to dmu, dscale, dquat, dopac, dsh.
 *   rgb: as in 3DGS (SH of the direction from the camera centre);
 *   ro_c = M (c - mu): dM += dro_c (c - mu)^T, dmu -= M^T dro_c;
 *   M_ij = R_ji / s_i: ds_i -= sum_j dM_ij M_ij / s_i, dR_ji += dM_ij / s_i;
 *   o' = o m, m = sqrt(det_0 / det): dopac = do' m, and m depends on Sigma_2D (UT):
 *     dm/ddet_0 = m / (2 det_0), dm/ddet = -m / (2 det), det_0 = c0 c2 - c1^2,
 *     det = (c0 + d)(c2 + d) - c1^2;
 *   Sigma_2D = sum_k wc_k (p_k - mu_2D)(p_k - mu_2D)^T, mu_2D = sum_k wm_k p_k;
 *   p_k = (fx x_k / z_k + cx, fy y_k / z_k + cy), (x_k, y_k, z_k) = W X_k + t;
 *   X_k = mu + sgn sqrt(3) s_a R[:, a]: dmu += dX_k, ds_a += sgn sqrt(3) R[:, a].dX_k,
 *     dR[:, a] += sgn sqrt(3) s_a dX_k;
 *   R = R(q / |q|) as in 3DGS. */
void oracle_project_ut_bwd(int64_t n, const double *mu, const double *scale, const double *quat, const double *opac,
                           const double *sh, const double *camv, const double *cfgv, const double *d_sd,
                           double *dmu, double *dscale, double *dquat, double *dopac, double *dsh) {
    ocam cam = read_cam(camv);
    ocfg cfg = read_cfg(cfgv);
    int K = (cfg.deg + 1) * (cfg.deg + 1);
    const double *V = cam.V;
    const double wm[7] = {0.0, 1.0 / 6, 1.0 / 6, 1.0 / 6, 1.0 / 6, 1.0 / 6, 1.0 / 6};
    const double wc[7] = {2.0, 1.0 / 6, 1.0 / 6, 1.0 / 6, 1.0 / 6, 1.0 / 6, 1.0 / 6};
    const double sq3 = sqrt(3.0);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        oproj_ut P;
        const double *D = d_sd + 16 * i;
        const double *s = scale + 3 * i;
        const double *m_ = mu + 3 * i;
        const double *shi = sh + (int64_t)3 * K * i;
        double *gmu = dmu + 3 * i, *gs = dscale + 3 * i, *gq = dquat + 4 * i, *gsh = dsh + (int64_t)3 * K * i;
        project_ut_one(m_, s, quat + 4 * i, opac[i], shi, &cam, &cfg, &P);
        memset(gmu, 0, 3 * sizeof(double));
        memset(gs, 0, 3 * sizeof(double));
        memset(gq, 0, 4 * sizeof(double));
        memset(gsh, 0, (size_t)3 * K * sizeof(double));
        dopac[i] = 0.0;
        if (!P.visible) continue;

        /* colour */
        double Y[16], dY[48];
        oracle_sh_basis(cfg.deg, P.dir, Y, dY);
        double gdir[3] = {0, 0, 0};
        for (int c = 0; c < 3; ++c) {
            if (!(P.raw[c] > 0.0)) continue;
            double g = D[13 + c];
            for (int k = 0; k < K; ++k) {
                gsh[3 * k + c] = Y[k] * g;
                for (int j = 0; j < 3; ++j) gdir[j] += g * shi[3 * k + c] * dY[3 * k + j];
            }
        }
        double dd = gdir[0] * P.dir[0] + gdir[1] * P.dir[1] + gdir[2] * P.dir[2];
        for (int j = 0; j < 3; ++j) gmu[j] += (gdir[j] - P.dir[j] * dd) / P.vlen;

        /* ro_c = M (c - mu) */
        double gM[9];
        for (int r = 0; r < 3; ++r)
            for (int j = 0; j < 3; ++j) gM[3 * r + j] = D[3 + 3 * r + j] + D[r] * (P.cp[j] - m_[j]);
        for (int j = 0; j < 3; ++j) gmu[j] -= P.M[j] * D[0] + P.M[3 + j] * D[1] + P.M[6 + j] * D[2];
        /* M_ij = R_ji / s_i */
        double gR[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
        for (int r = 0; r < 3; ++r)
            for (int j = 0; j < 3; ++j) {
                gs[r] -= gM[3 * r + j] * P.M[3 * r + j] / s[r];
                gR[3 * j + r] += gM[3 * r + j] / s[r];
            }

        /* o' = o m */
        dopac[i] = D[12] * P.mip;
        double gmip = D[12] * opac[i];
        double c0 = P.cov0[0], c1 = P.cov0[1], c2 = P.cov0[2], dil = cfg.dil;
        double kd0 = gmip * P.mip / (2.0 * P.det0), kd = -gmip * P.mip / (2.0 * P.det);
        double gc0 = kd0 * c2 + kd * (c2 + dil);
        double gc2 = kd0 * c0 + kd * (c0 + dil);
        double gc1 = -2.0 * c1 * (kd0 + kd);
        /* Sigma_2D from the projected sigma points */
        double gp[7][2], gbar[2] = {0.0, 0.0};
        for (int k = 0; k < 7; ++k) {
            double dx = P.pts[k][0] - P.mu2d[0], dy = P.pts[k][1] - P.mu2d[1];
            gp[k][0] = wc[k] * (2.0 * gc0 * dx + gc1 * dy);
            gp[k][1] = wc[k] * (gc1 * dx + 2.0 * gc2 * dy);
            gbar[0] -= gp[k][0];
            gbar[1] -= gp[k][1];
        }
        for (int k = 0; k < 7; ++k) {
            gp[k][0] += wm[k] * gbar[0];
            gp[k][1] += wm[k] * gbar[1];
        }
        for (int k = 0; k < 7; ++k) {
            double Jp[6];
            proj_jacobian(&cam, P.pc[k], Jp);
            double gpc[3] = {gp[k][0] * Jp[0] + gp[k][1] * Jp[3], gp[k][0] * Jp[1] + gp[k][1] * Jp[4],
                             gp[k][0] * Jp[2] + gp[k][1] * Jp[5]};
            double gX[3];
            for (int j = 0; j < 3; ++j) gX[j] = V[j] * gpc[0] + V[4 + j] * gpc[1] + V[8 + j] * gpc[2];
            for (int j = 0; j < 3; ++j) gmu[j] += gX[j];
            if (k == 0) continue;
            int a = (k - 1) / 2;
            double sgn = (k % 2) ? 1.0 : -1.0;
            gs[a] += sgn * sq3 * (P.R[a] * gX[0] + P.R[3 + a] * gX[1] + P.R[6 + a] * gX[2]);
            for (int j = 0; j < 3; ++j) gR[3 * j + a] += sgn * sq3 * s[a] * gX[j];
        }
        double dR[4][9];
        drot_dq(P.qn, dR);
        double gqn[4];
        for (int j = 0; j < 4; ++j) {
            double acc = 0.0;
            for (int e = 0; e < 9; ++e) acc += gR[e] * dR[j][e];
            gqn[j] = acc;
        }
        double dotq = gqn[0] * P.qn[0] + gqn[1] * P.qn[1] + gqn[2] * P.qn[2] + gqn[3] * P.qn[3];
        for (int j = 0; j < 4; ++j) gq[j] = (gqn[j] - P.qn[j] * dotq) / P.qnorm;
    }
}

/* ------------------------------------------------------------------------ */
/* LinPrim (Appendix, implementation of XPR-LinPrim; Listing LinPrim).       */
/* Octahedron {x : ||S^-1 R^T (x - mu)||_1 <= 1}, homogeneous density        */
/*   sigma = -log(1 - 0.99 o) / (2 min s),  o clipped to [0, 0.999].         */
/* Projection: m_c = W mu + t, d = |m_c|, mu_2D = (fx x/z + cx, fy y/z + cy), */
/* A = J3 W R diag(s) with J3 the pinhole Jacobian of (x_px, y_px) and a     */
/* third row d|m_c|/dm_c = m_c / d (Euclidean distance, so tau is depth     */
/* along the ray); c0, c1, c2 = rows of A^-1; slab normals                   */
/*   n_i = c0 + e1 c1 + e2 c2, (e1, e2) = (+,+), (+,-), (-,+), (-,-).        */
/* Extents: the largest pixel offsets of the six vertices, ex = max_k        */
/* |A_0k|, ey = max_k |A_1k|; the box of mu_2D - 0.5 as 3DGUT; depth = d.    */
/* Visible iff camera z > z_near, d > z_near, min s > 0, r > 0, tc > 0.      */
/* Evaluate at (x + 0.5, y + 0.5): slab i bounds tau to [m_i - h_i, m_i +    */
/* h_i], m_i = -(n_ix dX + n_iy dY) / n_iz, h_i = 1 / |n_iz| (|n_iz| <       */
/* 1e-10: no bound); dtau = min hi - max lo, alpha = 1 - exp(-sigma dtau)    */
/* when positive, else 0.  Tile cull: the per-tile bound of Eq.              */
/* (linprim_tile_cull) over the four pixel-centre corners of the tile.       */
/* Records: rec[12] with mu_2D [0,1], rgb [6..8], depth d [9], visible [11]; */
/* sd[16] = mu_2D (2), c0, c1, c2 (9), sigma, rgb (3), 0.                   */
/* ------------------------------------------------------------------------ */

#define LP_EPS 1e-10
#define LP_INF 1e10
static const double LP_E[4][2] = {{1, 1}, {1, -1}, {-1, 1}, {-1, -1}};

typedef struct {
    double mc[3], d, mu2d[2], J[9], M[9], A[9], Ai[9], n[4][3], ex, ey, sigma, smin, oc, rgb[3], raw[3], dir[3],
        vlen, qn[4], qnorm, R[9], pre[4];
    int kmin, oclip, bbox[4], tc, visible, front;
} oproj_lp;

static double det3(const double *A) {
    return A[0] * (A[4] * A[8] - A[5] * A[7]) - A[1] * (A[3] * A[8] - A[5] * A[6]) +
           A[2] * (A[3] * A[7] - A[4] * A[6]);
}

/* inverse by cofactors; returns the determinant */
static double inv3(const double *A, double *Ai) {
    double dt = det3(A);
    Ai[0] = (A[4] * A[8] - A[5] * A[7]) / dt;
    Ai[1] = (A[2] * A[7] - A[1] * A[8]) / dt;
    Ai[2] = (A[1] * A[5] - A[2] * A[4]) / dt;
    Ai[3] = (A[5] * A[6] - A[3] * A[8]) / dt;
    Ai[4] = (A[0] * A[8] - A[2] * A[6]) / dt;
    Ai[5] = (A[2] * A[3] - A[0] * A[5]) / dt;
    Ai[6] = (A[3] * A[7] - A[4] * A[6]) / dt;
    Ai[7] = (A[1] * A[6] - A[0] * A[7]) / dt;
    Ai[8] = (A[0] * A[4] - A[1] * A[3]) / dt;
    return dt;
}

static void project_lp_one(const double *mu, const double *s, const double *q, double o, const double *sh,
                           const ocam *cam, const ocfg *cfg, oproj_lp *P) {
    memset(P, 0, sizeof(*P));
    const double *V = cam->V;
    for (int i = 0; i < 3; ++i) P->mc[i] = V[4 * i] * mu[0] + V[4 * i + 1] * mu[1] + V[4 * i + 2] * mu[2] + V[4 * i + 3];
    quat_rot(q, P->qn, &P->qnorm, P->R);
    double cp[3];
    for (int i = 0; i < 3; ++i) cp[i] = -(V[i] * V[3] + V[4 + i] * V[7] + V[8 + i] * V[11]);
    double v[3] = {mu[0] - cp[0], mu[1] - cp[1], mu[2] - cp[2]};
    P->vlen = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
    for (int i = 0; i < 3; ++i) P->dir[i] = v[i] / P->vlen;
    int K = (cfg->deg + 1) * (cfg->deg + 1);
    double Y[16];
    oracle_sh_basis(cfg->deg, P->dir, Y, NULL);
    for (int c = 0; c < 3; ++c) {
        double acc = 0.5;
        for (int k = 0; k < K; ++k) acc += sh[3 * k + c] * Y[k];
        P->raw[c] = acc;
        P->rgb[c] = acc > 0.0 ? acc : 0.0;
    }
    P->kmin = 0;
    for (int k = 1; k < 3; ++k)
        if (s[k] < s[P->kmin]) P->kmin = k;
    P->smin = s[P->kmin];
    P->oc = o < 0.0 ? 0.0 : (o > 0.999 ? 0.999 : o);
    P->oclip = !(o > 0.0 && o < 0.999);
    P->sigma = -log1p(-0.99 * P->oc) / (2.0 * P->smin);
    const double x = P->mc[0], y = P->mc[1], z = P->mc[2];
    P->d = sqrt(x * x + y * y + z * z);
    P->front = (z > cam->z_near) && (P->d > cam->z_near) && (P->smin > 0.0);
    if (!P->front) return;
    P->mu2d[0] = cam->fx * x / z + cam->cx;
    P->mu2d[1] = cam->fy * y / z + cam->cy;
    double J[9] = {cam->fx / z, 0.0, -cam->fx * x / (z * z), 0.0, cam->fy / z, -cam->fy * y / (z * z),
                   x / P->d, y / P->d, z / P->d};
    memcpy(P->J, J, sizeof(J));
    for (int i = 0; i < 3; ++i)
        for (int k = 0; k < 3; ++k)
            P->M[3 * i + k] = V[4 * i] * P->R[k] + V[4 * i + 1] * P->R[3 + k] + V[4 * i + 2] * P->R[6 + k];
    for (int i = 0; i < 3; ++i)
        for (int k = 0; k < 3; ++k)
            P->A[3 * i + k] = (J[3 * i] * P->M[k] + J[3 * i + 1] * P->M[3 + k] + J[3 * i + 2] * P->M[6 + k]) * s[k];
    inv3(P->A, P->Ai);
    for (int i = 0; i < 4; ++i)
        for (int c = 0; c < 3; ++c)
            P->n[i][c] = P->Ai[c] + LP_E[i][0] * P->Ai[3 + c] + LP_E[i][1] * P->Ai[6 + c];
    P->ex = fmax(fabs(P->A[0]), fmax(fabs(P->A[1]), fabs(P->A[2])));
    P->ey = fmax(fabs(P->A[3]), fmax(fabs(P->A[4]), fabs(P->A[5])));
    double r = P->ex > P->ey ? P->ex : P->ey;
    int Wt = (cam->W + cfg->tw - 1) / cfg->tw, Ht = (cam->H + cfg->th - 1) / cfg->th;
    P->pre[0] = (P->mu2d[0] - 0.5 - P->ex) / cfg->tw;
    P->pre[1] = (P->mu2d[1] - 0.5 - P->ey) / cfg->th;
    P->pre[2] = (P->mu2d[0] - 0.5 + P->ex) / cfg->tw;
    P->pre[3] = (P->mu2d[1] - 0.5 + P->ey) / cfg->th;
    P->bbox[0] = (int)clampd(floor(P->pre[0]), 0.0, (double)Wt);
    P->bbox[1] = (int)clampd(floor(P->pre[1]), 0.0, (double)Ht);
    P->bbox[2] = (int)clampd(floor(P->pre[2]) + 1.0, 0.0, (double)Wt);
    P->bbox[3] = (int)clampd(floor(P->pre[3]) + 1.0, 0.0, (double)Ht);
    int tc = (P->bbox[2] - P->bbox[0]) * (P->bbox[3] - P->bbox[1]);
    P->visible = (r > 0.0) && (tc > 0);
    P->tc = P->visible ? tc : 0;
    if (!P->visible) memset(P->bbox, 0, sizeof(P->bbox));
}

void oracle_project_lp(int64_t n, const double *mu, const double *scale, const double *quat, const double *opac,
                       const double *sh, const double *camv, const double *cfgv, double *rec, double *sd,
                       int32_t *bbox, int32_t *tc, double *pre, double *aux) {
    ocam cam = read_cam(camv);
    ocfg cfg = read_cfg(cfgv);
    int K = (cfg.deg + 1) * (cfg.deg + 1);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        oproj_lp P;
        project_lp_one(mu + 3 * i, scale + 3 * i, quat + 4 * i, opac[i], sh + (int64_t)3 * K * i, &cam, &cfg, &P);
        double *r = rec + 12 * i, *d = sd + 16 * i;
        memset(r, 0, 12 * sizeof(double));
        memset(d, 0, 16 * sizeof(double));
        r[9] = P.d;
        if (P.visible) {
            r[0] = P.mu2d[0];
            r[1] = P.mu2d[1];
            for (int c = 0; c < 3; ++c) r[6 + c] = P.rgb[c];
            r[11] = 1.0;
            d[0] = P.mu2d[0];
            d[1] = P.mu2d[1];
            for (int k = 0; k < 9; ++k) d[2 + k] = P.Ai[k];
            d[11] = P.sigma;
            for (int c = 0; c < 3; ++c) d[12 + c] = P.rgb[c];
        }
        for (int j = 0; j < 4; ++j) bbox[4 * i + j] = P.bbox[j];
        tc[i] = P.tc;
        if (pre)
            for (int j = 0; j < 4; ++j) pre[4 * i + j] = P.visible ? P.pre[j] : 0.0;
        if (aux) { /* A (9), ex, ey, camera z */
            for (int k = 0; k < 9; ++k) aux[12 * i + k] = P.A[k];
            aux[12 * i + 9] = P.ex;
            aux[12 * i + 10] = P.ey;
            aux[12 * i + 11] = P.mc[2];
        }
    }
}

/* slab normals of paper-form shader data */
static void lp_normals(const double *S, double n[4][3]) {
    for (int i = 0; i < 4; ++i)
        for (int c = 0; c < 3; ++c) n[i][c] = S[2 + c] + LP_E[i][0] * S[5 + c] + LP_E[i][1] * S[8 + c];
}

/* chord dtau of the slab intersection at pixel-centre offset (dX, dY); lo / hi receive the binding
 * slabs (may be NULL) */
static double lp_chord(const double n[4][3], double dX, double dY, int *lo_i, int *hi_i) {
    double enter = -INFINITY, exit_ = INFINITY;
    int li = -1, hj = -1;
    for (int i = 0; i < 4; ++i) {
        if (!(fabs(n[i][2]) >= LP_EPS)) continue;
        double m = -(n[i][0] * dX + n[i][1] * dY) / n[i][2], h = 1.0 / fabs(n[i][2]);
        if (m - h > enter) {
            enter = m - h;
            li = i;
        }
        if (m + h < exit_) {
            exit_ = m + h;
            hj = i;
        }
    }
    if (lo_i) *lo_i = li;
    if (hi_i) *hi_i = hj;
    return (enter < exit_) ? exit_ - enter : 0.0;
}

double oracle_lp_chord(const double *sd, double dX, double dY) {
    double n[4][3];
    lp_normals(sd, n);
    return lp_chord(n, dX, dY, NULL, NULL);
}

/* The per-tile bound of Eq. (linprim_tile_cull) at pixel-centre corners X in {x0, x1}, Y in {y0, y1}. */
static double lp_tile_bound(const double n[4][3], double mx, double my, double x0, double y0, double x1, double y1) {
    double mc[4][4], half[4];
    const double cx[4] = {x0, x0, x1, x1}, cy[4] = {y0, y1, y0, y1};
    for (int i = 0; i < 4; ++i) {
        int ok = fabs(n[i][2]) >= LP_EPS;
        double inv = ok ? 1.0 / n[i][2] : 0.0;
        half[i] = ok ? fabs(inv) : LP_INF;
        for (int c = 0; c < 4; ++c) mc[i][c] = -inv * (n[i][0] * (cx[c] - mx) + n[i][1] * (cy[c] - my));
    }
    double best = INFINITY;
    for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j) {
            double g = -INFINITY;
            for (int c = 0; c < 4; ++c) g = fmax(g, mc[i][c] - mc[j][c]);
            g += half[i] + half[j];
            if (g < best) best = g;
        }
    return best > 0.0 ? best : 0.0;
}

/* The kernels' FP32 cull decision on their shader data s32[20]: mu_2D (2), sigma, -log(1 -
 * alpha_t), then per slab (p, q, h) = (n_x / n_z, n_y / n_z, 1 / |n_z|) (p = q = 0, h = inf when
 * |n_z| < 1e-10); one correctly rounded IEEE operation per step in this order, no FMA. */
static int lp_keep_f32(const float *s32, float X0, float Y0, float X1, float Y1) {
    const float mx = s32[0], my = s32[1], sigma = s32[2], req = s32[3];
    const float dX[2] = {X0 - mx, X1 - mx}, dY[2] = {Y0 - my, Y1 - my};
    float m[4][4], h[4];
    for (int i = 0; i < 4; ++i) {
        const float p = s32[4 + 3 * i], qq = s32[5 + 3 * i];
        h[i] = s32[6 + 3 * i];
        for (int c = 0; c < 4; ++c) {
            float t = p * dX[c >> 1];
            float u = qq * dY[c & 1];
            float w = t + u;
            m[i][c] = -w;
        }
    }
    float best = INFINITY;
    for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j) {
            float g = m[i][0] - m[j][0];
            for (int c = 1; c < 4; ++c) {
                float e = m[i][c] - m[j][c];
                g = fmaxf(g, e);
            }
            g = g + h[i];
            g = g + h[j];
            best = fminf(best, g);
        }
    best = fmaxf(best, 0.0f);
    float a = sigma * best;
    return a >= req;
}

/* tile bounds for LinPrim: the corners' pixel centres (inclusive pixel bounds + 0.5) */
static void lp_tile_corners(int tx, int ty, const ocam *cam, const ocfg *cfg, double *c) {
    int x0 = tx * cfg->tw, y0 = ty * cfg->th;
    int x1 = x0 + cfg->tw - 1, y1 = y0 + cfg->th - 1;
    if (x1 > cam->W - 1) x1 = cam->W - 1;
    if (y1 > cam->H - 1) y1 = cam->H - 1;
    c[0] = x0 + 0.5;
    c[1] = y0 + 0.5;
    c[2] = x1 + 0.5;
    c[3] = y1 + 0.5;
}

int oracle_lp_keep(const double *sd, int tx, int ty, const double *camv, const double *cfgv) {
    ocam cam = read_cam(camv);
    ocfg cfg = read_cfg(cfgv);
    double n[4][3], c[4];
    lp_normals(sd, n);
    lp_tile_corners(tx, ty, &cam, &cfg, c);
    double req = -log1p(-cfg.at);
    return sd[11] * lp_tile_bound(n, sd[0], sd[1], c[0], c[1], c[2], c[3]) >= req;
}

double oracle_lp_tile_bound(const double *sd, int tx, int ty, const double *camv, const double *cfgv) {
    ocam cam = read_cam(camv);
    ocfg cfg = read_cfg(cfgv);
    double n[4][3], c[4];
    lp_normals(sd, n);
    lp_tile_corners(tx, ty, &cam, &cfg, c);
    return lp_tile_bound(n, sd[0], sd[1], c[0], c[1], c[2], c[3]);
}

/* Binning for LinPrim (as oracle_bin): exact32 != 0 takes the FP32 decision on kernel-form shader
 * data sd32[n*20] and depths from rec32; else the FP64 bound on paper-form sd64[n*16] with the
 * depth keys key[n] (NULL = rec64's depth rounded to float32). */
int64_t oracle_bin_lp(int64_t n, const double *rec64, const double *sd64, const float *rec32, const float *sd32,
                      const float *key, const int32_t *bbox, const double *camv, const double *cfgv, int exact32,
                      const int64_t *order, int32_t *counts, uint64_t *keys, uint32_t *vals) {
    ocam cam = read_cam(camv);
    ocfg cfg = read_cfg(cfgv);
    int Wt = (cam.W + cfg.tw - 1) / cfg.tw;
    double req = -log1p(-cfg.at);
    int64_t total = 0;
    for (int64_t pos = 0; pos < n; ++pos) {
        int64_t i = order ? order[pos] : pos;
        const int32_t *bb = bbox + 4 * i;
        int w = bb[2] - bb[0], h = bb[3] - bb[1];
        int tc = (w > 0 && h > 0) ? w * h : 0;
        int cnt = 0;
        double nn[4][3];
        if (!exact32 && tc > 0) lp_normals(sd64 + 16 * i, nn);
        for (int r = 0; r < tc; ++r) {
            int tx = bb[0] + r % w, ty = bb[1] + r / w;
            double c[4];
            lp_tile_corners(tx, ty, &cam, &cfg, c);
            int keep;
            float depth32;
            if (exact32) {
                keep = lp_keep_f32(sd32 + 20 * i, (float)c[0], (float)c[1], (float)c[2], (float)c[3]);
                depth32 = rec32[12 * i + 9];
            } else {
                const double *S = sd64 + 16 * i;
                keep = S[11] * lp_tile_bound(nn, S[0], S[1], c[0], c[1], c[2], c[3]) >= req;
                depth32 = key ? key[i] : (float)rec64[12 * i + 9];
            }
            if (!keep) continue;
            if (keys) {
                keys[total] = ((uint64_t)(uint32_t)(ty * Wt + tx) << 32) | (uint64_t)f32_bits(depth32);
                vals[total] = (uint32_t)i;
            }
            ++total;
            ++cnt;
        }
        if (counts) counts[pos] = cnt;
    }
    return total;
}

typedef struct {
    int64_t idx;
    double alpha, T, dt, e;
    int clamped, lo, hi;
    double dX, dY;
} contrib_lp;

/* the compositing walk of the framework with the LinPrim evaluate (valid = 1) */
static int walk_lp(double X, double Y, const double *sd, const int64_t *list, int len, const ocfg *cfg, double delta,
                   double C[3], double *Tout, int *last, int *band, double *jump, contrib_lp *out, uint64_t *sig) {
    double T = 1.0, eT = 0.0, J = 0.0;
    C[0] = C[1] = C[2] = 0.0;
    int nc = 0, bd = 0;
    uint64_t hsh = sig ? *sig : 0;
    *last = 0;
    for (int k = 0; k < len; ++k) {
        const double *S = sd + 16 * list[k];
        double n[4][3];
        lp_normals(S, n);
        double dX = X - S[0], dY = Y - S[1];
        int lo, hi;
        double dt = lp_chord(n, dX, dY, &lo, &hi);
        double e = exp(-S[11] * dt);
        double a0 = dt > 0.0 ? 1.0 - e : 0.0;
        double alpha = a0 < cfg->amax ? a0 : cfg->amax;
        if (delta > 0.0 && fabs(a0 - cfg->amax) <= delta * cfg->amax) bd |= 2;
        if (delta > 0.0 && fabs(alpha - cfg->at) <= delta * cfg->at) {
            double am = alpha > cfg->at ? alpha : cfg->at;
            bd |= 1;
            J += 2.0 * am * T;
            eT += am / (1.0 - am);
        }
        if (alpha < cfg->at) continue;
        double tt = T * (1.0 - alpha);
        if (delta > 0.0 && fabs(log(tt / cfg->teps)) <= eT + alpha * delta / (1.0 - alpha) + delta) {
            bd |= 1;
            J += T;
        }
        if (tt < cfg->teps) {
            hsh = hsh * 1099511628211ULL ^ 0xffffULL;
            break;
        }
        if (out) {
            contrib_lp *c = out + nc;
            c->idx = list[k];
            c->alpha = alpha;
            c->T = T;
            c->dt = dt;
            c->e = e;
            c->clamped = !(a0 < cfg->amax);
            c->lo = lo;
            c->hi = hi;
            c->dX = dX;
            c->dY = dY;
        }
        hsh = (hsh ^ (uint64_t)(list[k] + 1)) * 1099511628211ULL;
        hsh = (hsh ^ (uint64_t)(4 * lo + hi + 17)) * 1099511628211ULL;
        for (int c = 0; c < 3; ++c) C[c] += S[12 + c] * alpha * T;
        T = tt;
        eT += alpha * delta / (1.0 - alpha) + delta;
        ++nc;
        *last = k + 1;
    }
    for (int c = 0; c < 3; ++c) C[c] += T * cfg->bg[c];
    *Tout = T;
    *band = bd;
    if (jump) *jump = J;
    if (sig) *sig = hsh;
    return nc;
}

void oracle_render_tiles_lp(int64_t n, const double *sd, const uint32_t *vals, const int32_t *ranges,
                            const double *camv, const double *cfgv, double delta, double *image, double *tfinal,
                            int32_t *ncontrib, int32_t *band, double *jump, uint64_t *psig) {
    (void)n;
    ocam cam = read_cam(camv);
    ocfg cfg = read_cfg(cfgv);
    int Wt = (cam.W + cfg.tw - 1) / cfg.tw, Ht = (cam.H + cfg.th - 1) / cfg.th;
    int64_t HW = (int64_t)cam.W * cam.H;
#pragma omp parallel for schedule(dynamic, 1)
    for (int t = 0; t < Wt * Ht; ++t) {
        int tx = t % Wt, ty = t / Wt;
        int s0 = ranges[2 * t], e0 = ranges[2 * t + 1];
        int len = e0 - s0;
        int64_t *list = (int64_t *)malloc((size_t)(len > 0 ? len : 1) * sizeof(int64_t));
        for (int k = 0; k < len; ++k) list[k] = vals[s0 + k];
        for (int yy = 0; yy < cfg.th; ++yy)
            for (int xx = 0; xx < cfg.tw; ++xx) {
                int x = tx * cfg.tw + xx, y = ty * cfg.th + yy;
                if (x >= cam.W || y >= cam.H) continue;
                double C[3], T, J;
                int last, bd;
                uint64_t h = 0;
                walk_lp(x + 0.5, y + 0.5, sd, list, len, &cfg, delta, C, &T, &last, &bd, &J, NULL, &h);
                int64_t p = (int64_t)y * cam.W + x;
                if (jump) jump[p] = J;
                for (int c = 0; c < 3; ++c) image[c * HW + p] = C[c];
                tfinal[p] = T;
                ncontrib[p] = last;
                band[p] = bd;
                if (psig) psig[p] = h;
            }
        free(list);
    }
}

/* Adjoint of the LinPrim walk: dtau = (m_hi + h_hi) - (m_lo - h_lo) for the binding slabs, with
 * m = -(n_x dX + n_y dY) / n_z and h = 1 / |n_z|:
 *   dm/dn_x = -dX / n_z, dm/dn_y = -dY / n_z, dm/dn_z = -m / n_z, dh/dn_z = -h / n_z,
 *   dm/dmu_x = n_x / n_z, dm/dmu_y = n_y / n_z;
 * alpha = 1 - exp(-sigma dtau): dalpha/dsigma = dtau e, dalpha/ddtau = sigma e (nothing through the
 * clamp); n_i = c0 + e1 c1 + e2 c2.  d_sd[n*16] in the paper-form layout. */
static void pixel_adjoint_lp(const double *sd, const contrib_lp *cs, int nc, double Tfin, const double *g,
                             const ocfg *cfg, double *d_sd) {
    if (nc == 0) return;
    double *S = (double *)malloc((size_t)nc * 3 * sizeof(double));
    for (int c = 0; c < 3; ++c) {
        double acc = Tfin * cfg->bg[c];
        for (int i = nc - 1; i >= 0; --i) {
            S[3 * i + c] = acc;
            acc += sd[16 * cs[i].idx + 12 + c] * cs[i].alpha * cs[i].T;
        }
    }
    for (int i = 0; i < nc; ++i) {
        const double *Sd = sd + 16 * cs[i].idx;
        double *D = d_sd + 16 * cs[i].idx;
        double a = cs[i].alpha, T = cs[i].T;
        double da = 0.0;
        for (int c = 0; c < 3; ++c) {
            D[12 + c] += g[c] * a * T;
            da += g[c] * (Sd[12 + c] * T - S[3 * i + c] / (1.0 - a));
        }
        if (cs[i].clamped) continue;
        D[11] += da * cs[i].dt * cs[i].e;
        double gdt = da * Sd[11] * cs[i].e;
        double n[4][3];
        lp_normals(Sd, n);
        for (int side = 0; side < 2; ++side) {
            int k = side == 0 ? cs[i].hi : cs[i].lo;
            double gm = side == 0 ? gdt : -gdt, gh = gdt;
            const double *nk = n[k];
            double m = -(nk[0] * cs[i].dX + nk[1] * cs[i].dY) / nk[2], h = 1.0 / fabs(nk[2]);
            double gn[3] = {gm * (-cs[i].dX / nk[2]), gm * (-cs[i].dY / nk[2]), gm * (-m / nk[2]) + gh * (-h / nk[2])};
            D[0] += gm * nk[0] / nk[2];
            D[1] += gm * nk[1] / nk[2];
            for (int c = 0; c < 3; ++c) {
                D[2 + c] += gn[c];
                D[5 + c] += LP_E[k][0] * gn[c];
                D[8 + c] += LP_E[k][1] * gn[c];
            }
        }
    }
    free(S);
}

void oracle_render_bwd_tiles_lp(int64_t n, const double *sd, const uint32_t *vals, const int32_t *ranges,
                                const double *camv, const double *cfgv, const double *d_image, double *d_sd) {
    ocam cam = read_cam(camv);
    ocfg cfg = read_cfg(cfgv);
    int Wt = (cam.W + cfg.tw - 1) / cfg.tw, Ht = (cam.H + cfg.th - 1) / cfg.th;
    int64_t HW = (int64_t)cam.W * cam.H;
    memset(d_sd, 0, (size_t)n * 16 * sizeof(double));
    for (int t = 0; t < Wt * Ht; ++t) {
        int tx = t % Wt, ty = t / Wt;
        int s0 = ranges[2 * t], e0 = ranges[2 * t + 1];
        int len = e0 - s0;
        if (len <= 0) continue;
        int64_t *list = (int64_t *)malloc((size_t)len * sizeof(int64_t));
        contrib_lp *cs = (contrib_lp *)malloc((size_t)len * sizeof(contrib_lp));
        for (int k = 0; k < len; ++k) list[k] = vals[s0 + k];
        for (int yy = 0; yy < cfg.th; ++yy)
            for (int xx = 0; xx < cfg.tw; ++xx) {
                int x = tx * cfg.tw + xx, y = ty * cfg.th + yy;
                if (x >= cam.W || y >= cam.H) continue;
                int64_t p = (int64_t)y * cam.W + x;
                double g[3] = {d_image[p], d_image[HW + p], d_image[2 * HW + p]};
                if (g[0] == 0.0 && g[1] == 0.0 && g[2] == 0.0) continue;
                double C[3], T;
                int last, bd;
                int nc = walk_lp(x + 0.5, y + 0.5, sd, list, len, &cfg, 0.0, C, &T, &last, &bd, NULL, cs, NULL);
                pixel_adjoint_lp(sd, cs, nc, T, g, &cfg, d_sd);
            }
        free(cs);
        free(list);
    }
}

/* Adjoint of the LinPrim projection from paper-form d_sd (dmu_2D, dc0, dc1, dc2, dsigma, drgb):
 *   A^-1 rows c_k: dA = -A^-T dA^-1 A^-T;  A = J3 M diag(s), M = W R:
 *     dJ3 = dA (M diag(s))^T, dM = J3^T dA diag(s), ds_k += sum_i dA_ik (J3 M)_ik, dR = W^T dM;
 *   J3(m_c): J00 = fx/z, J02 = -fx x/z^2, J11 = fy/z, J12 = -fy y/z^2, J2k = m_c,k / d;
 *   mu_2D(m_c); m_c = W mu + t;
 *   sigma = -log(1 - 0.99 o) / (2 s_min): dsigma/do = 0.99 / ((1 - 0.99 o) 2 s_min) (0 where o is
 *   clipped), dsigma/ds_min = -sigma / s_min;  colour as in 3DGS. */
void oracle_project_lp_bwd(int64_t n, const double *mu, const double *scale, const double *quat, const double *opac,
                           const double *sh, const double *camv, const double *cfgv, const double *d_sd,
                           double *dmu, double *dscale, double *dquat, double *dopac, double *dsh) {
    ocam cam = read_cam(camv);
    ocfg cfg = read_cfg(cfgv);
    int K = (cfg.deg + 1) * (cfg.deg + 1);
    const double *V = cam.V;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        oproj_lp P;
        const double *D = d_sd + 16 * i;
        const double *s = scale + 3 * i;
        const double *shi = sh + (int64_t)3 * K * i;
        double *gmu = dmu + 3 * i, *gs = dscale + 3 * i, *gq = dquat + 4 * i, *gsh = dsh + (int64_t)3 * K * i;
        project_lp_one(mu + 3 * i, s, quat + 4 * i, opac[i], shi, &cam, &cfg, &P);
        memset(gmu, 0, 3 * sizeof(double));
        memset(gs, 0, 3 * sizeof(double));
        memset(gq, 0, 4 * sizeof(double));
        memset(gsh, 0, (size_t)3 * K * sizeof(double));
        dopac[i] = 0.0;
        if (!P.visible) continue;
        /* colour */
        double Y[16], dY[48];
        oracle_sh_basis(cfg.deg, P.dir, Y, dY);
        double gdir[3] = {0, 0, 0};
        for (int c = 0; c < 3; ++c) {
            if (!(P.raw[c] > 0.0)) continue;
            double g = D[12 + c];
            for (int k = 0; k < K; ++k) {
                gsh[3 * k + c] = Y[k] * g;
                for (int j = 0; j < 3; ++j) gdir[j] += g * shi[3 * k + c] * dY[3 * k + j];
            }
        }
        double dd = gdir[0] * P.dir[0] + gdir[1] * P.dir[1] + gdir[2] * P.dir[2];
        for (int j = 0; j < 3; ++j) gmu[j] += (gdir[j] - P.dir[j] * dd) / P.vlen;
        /* sigma */
        if (!P.oclip) dopac[i] = D[11] * 0.99 / ((1.0 - 0.99 * P.oc) * 2.0 * P.smin);
        gs[P.kmin] += D[11] * (-P.sigma / P.smin);
        /* A^-1 -> A */
        const double *Ai = P.Ai;
        double G[9], T1[9], dA[9];
        for (int k = 0; k < 9; ++k) G[k] = D[2 + k];
        /* dA = -Ai^T G Ai^T */
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) {
                double acc = 0.0;
                for (int k = 0; k < 3; ++k) acc += Ai[3 * k + a] * G[3 * k + b];
                T1[3 * a + b] = acc;
            }
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) {
                double acc = 0.0;
                for (int k = 0; k < 3; ++k) acc += T1[3 * a + k] * Ai[3 * b + k];
                dA[3 * a + b] = -acc;
            }
        /* A = J M diag(s) */
        double JM[9];
        for (int a = 0; a < 3; ++a)
            for (int k = 0; k < 3; ++k)
                JM[3 * a + k] = P.J[3 * a] * P.M[k] + P.J[3 * a + 1] * P.M[3 + k] + P.J[3 * a + 2] * P.M[6 + k];
        double dJ[9], dM[9];
        for (int a = 0; a < 3; ++a)
            for (int l = 0; l < 3; ++l) {
                double acc = 0.0;
                for (int k = 0; k < 3; ++k) acc += dA[3 * a + k] * P.M[3 * l + k] * s[k];
                dJ[3 * a + l] = acc;
            }
        for (int l = 0; l < 3; ++l)
            for (int k = 0; k < 3; ++k) {
                double acc = 0.0;
                for (int a = 0; a < 3; ++a) acc += P.J[3 * a + l] * dA[3 * a + k];
                dM[3 * l + k] = acc * s[k];
            }
        for (int k = 0; k < 3; ++k)
            for (int a = 0; a < 3; ++a) gs[k] += dA[3 * a + k] * JM[3 * a + k];
        double gR[9];
        for (int a = 0; a < 3; ++a)
            for (int k = 0; k < 3; ++k) gR[3 * a + k] = V[a] * dM[k] + V[4 + a] * dM[3 + k] + V[8 + a] * dM[6 + k];
        /* J(m_c) and mu_2D(m_c) */
        const double x = P.mc[0], y = P.mc[1], z = P.mc[2], d = P.d;
        double gmc[3] = {0, 0, 0};
        gmc[2] += dJ[0] * (-cam.fx / (z * z));
        gmc[0] += dJ[2] * (-cam.fx / (z * z));
        gmc[2] += dJ[2] * (2.0 * cam.fx * x / (z * z * z));
        gmc[2] += dJ[4] * (-cam.fy / (z * z));
        gmc[1] += dJ[5] * (-cam.fy / (z * z));
        gmc[2] += dJ[5] * (2.0 * cam.fy * y / (z * z * z));
        for (int k = 0; k < 3; ++k)
            for (int l = 0; l < 3; ++l) gmc[l] += dJ[6 + k] * ((k == l ? 1.0 / d : 0.0) - P.mc[k] * P.mc[l] / (d * d * d));
        gmc[0] += D[0] * cam.fx / z;
        gmc[1] += D[1] * cam.fy / z;
        gmc[2] += -(D[0] * cam.fx * x + D[1] * cam.fy * y) / (z * z);
        for (int j = 0; j < 3; ++j) gmu[j] += V[j] * gmc[0] + V[4 + j] * gmc[1] + V[8 + j] * gmc[2];
        double dRq[4][9];
        drot_dq(P.qn, dRq);
        double gqn[4];
        for (int j = 0; j < 4; ++j) {
            double acc = 0.0;
            for (int e = 0; e < 9; ++e) acc += gR[e] * dRq[j][e];
            gqn[j] = acc;
        }
        double dotq = gqn[0] * P.qn[0] + gqn[1] * P.qn[1] + gqn[2] * P.qn[2] + gqn[3] * P.qn[3];
        for (int j = 0; j < 4; ++j) gq[j] = (gqn[j] - P.qn[j] * dotq) / P.qnorm;
    }
}

int oracle_abi_version(void) { return 5; }
