/*
 * FP64 CPU oracle for ConeGaussian's anti-aliased ray-Gaussian render.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or
 * call this file; only tests/, the smoke check and the benchmark's CPU
 * baseline use it.  It shares no code, header, table or constant generator
 * with the CUDA library: every formula here is written out again from the
 * paper, in double precision, in the paper's order and notation.
 *
 * What it computes (per pixel, per Gaussian, then compositing):
 *   rays      d = Pi^-1(p), d_i = Pi^-1(p + Delta_i), Delta_x=(1/2,0),
 *             Delta_y=(0,1/2)                               (Sec. 4.1, Eq. 5-6)
 *   whitening W = S^-1 R^T, o_u = W(o-mu), d_u = W d        (Sec. 3, Eq. 1)
 *   t*        = -<o_u,d_u>/|d_u|^2, q = M_perp o_u          (Eq. 2)
 *   e_i       = t* M_perp W (d_i - d)                       (Eq. 6)
 *   Sigma_fp  = (e_x e_x^T + e_y e_y^T)/3                   (Eq. 8)
 *   floor     Sigma_eff = Sigma + rho^2 I,
 *             sigma_eff = sigma prod s_i/sqrt(s_i^2+rho^2)  (Eq. 10)
 *   marginal  Sigma_render = W [W^-1 Sigma_fp W^-T - rho^2 I]_+ W^T  (Eq. 12)
 *             (literal 3x3 form: Jacobi eigen-decomposition, clamp, re-whiten)
 *   response  T = sigma_eff det(A)^-1/2 exp(-q^T A^-1 q / 2),
 *             A = I + Sigma_render, symmetric, A >= I: det A and
 *             q^T A^-1 q from its eigen-decomposition      (Eq. 9)
 *   blend     c = sum_k c_k a_k prod_{j<k}(1-a_j), sorted by depth (Eq. 4)
 *   floor rho^2 = min_v tr(Sigma_fp^(v))/2 at the Gaussian-centre pixel (Eq. 11)
 *
 * Readings where the paper is silent (stated once here, used throughout):
 *   - Eq. 9 drops the longitudinal factor C[w] of Eq. 3: C = 1, so the
 *     footprint -> 0 limit is sigma e^{-D^2/2}.
 *   - compositing follows the usual 3DGS conventions: a = min(0.99, T);
 *     pairs with a < 1/255 are skipped; the walk stops before pair k when
 *     T_acc (1 - a_k) < 1e-4; background is 0.
 *   - pairs with t* <= 0.01 (behind / at the optical centre) are skipped.
 *   - the per-ray depth order uses the Gaussian key |mu - o| (the t* of the
 *     ray through mu), ties broken by Gaussian index; like the valid mask,
 *     this integer decision is taken in FP32 by a fixed operation sequence
 *     so that every implementation orders pairs identically.
 *   - KB fisheye: theta_d = theta (1 + k1 th^2 + k2 th^4 + k3 th^6 + k4 th^8),
 *     pixel valid iff its normalised radius is inside theta_d(theta_lim);
 *     an edge ray that leaves the valid disc is replaced by the backward
 *     difference d - Pi^-1(p - Delta_i).
 *   - SH colour: real SH to degree 3 (positive-constant real basis, l-major,
 *     m = -l..l), direction (mu - o)/|mu - o|, colour = max(0, SH + 1/2).
 *
 * The FP32 section at the end emulates the conservative angular-tile binning
 * rule: the rule is a definition of this library (the paper has no binning),
 * written as a fixed sequence of correctly rounded FP32 operations so that
 * pair counts can be compared bit for bit.  It is compiled with
 * -ffp-contract=off so no operation is fused.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#define ALPHA_MIN (1.0 / 255.0)
#define ALPHA_MAX 0.99
#define T_STOP 1e-4
#define T_NEAR 0.01
#define UT_TILE 8   /* tile side of the UT gate (pixels) */

/* ------------------------------------------------------------------ camera */

/* Packed camera (24 doubles):
 * [0] model (0 pinhole, 1 KB)  [1] width  [2] height
 * [3..6] fx fy cx cy           [7..10] k1..k4
 * [11..19] R (camera->world rotation, row-major)  [20..22] o  [23] theta_lim */
typedef struct {
    int model, W, H;
    double fx, fy, cx, cy, k[4], R[9], Rinv[9], o[3], thlim;
} ocam;

static void unpack_cam(const double *p, ocam *c) {
    c->model = (int)p[0];
    c->W = (int)p[1];
    c->H = (int)p[2];
    c->fx = p[3]; c->fy = p[4]; c->cx = p[5]; c->cy = p[6];
    for (int i = 0; i < 4; ++i) c->k[i] = p[7 + i];
    for (int i = 0; i < 9; ++i) c->R[i] = p[11 + i];
    for (int i = 0; i < 3; ++i) c->o[i] = p[20 + i];
    c->thlim = p[23];
    /* exact inverse of the given (FP32-rounded, nearly orthonormal) rotation */
    const double *R = c->R;
    double det = R[0] * (R[4] * R[8] - R[5] * R[7]) - R[1] * (R[3] * R[8] - R[5] * R[6]) +
                 R[2] * (R[3] * R[7] - R[4] * R[6]);
    c->Rinv[0] = (R[4] * R[8] - R[5] * R[7]) / det;
    c->Rinv[1] = (R[2] * R[7] - R[1] * R[8]) / det;
    c->Rinv[2] = (R[1] * R[5] - R[2] * R[4]) / det;
    c->Rinv[3] = (R[5] * R[6] - R[3] * R[8]) / det;
    c->Rinv[4] = (R[0] * R[8] - R[2] * R[6]) / det;
    c->Rinv[5] = (R[2] * R[3] - R[0] * R[5]) / det;
    c->Rinv[6] = (R[3] * R[7] - R[4] * R[6]) / det;
    c->Rinv[7] = (R[1] * R[6] - R[0] * R[7]) / det;
    c->Rinv[8] = (R[0] * R[4] - R[1] * R[3]) / det;
}

/* FP32 validity rule (shared decision, taken in FP32 on both sides). */
static int f32_valid_xy(const ocam *c, double xd, double yd) {
    if (c->model == 0) return 1;
    float x = (float)xd, y = (float)yd;
    float fx = (float)c->fx, fy = (float)c->fy, cx = (float)c->cx, cy = (float)c->cy;
    float k0 = (float)c->k[0], k1 = (float)c->k[1], k2 = (float)c->k[2], k3 = (float)c->k[3];
    float th = (float)c->thlim;
    float t2 = th * th;
    float p = ((k3 * t2 + k2) * t2 + k1) * t2 + k0;
    float rl = th * (1.0f + t2 * p);
    float rl2 = rl * rl;
    float a = (x - cx) / fx;
    float b = (y - cy) / fy;
    float r2 = a * a + b * b;
    return r2 <= rl2;
}

static double kb_thd(const double *k, double th) {
    double t2 = th * th;
    return th * (1.0 + t2 * (k[0] + t2 * (k[1] + t2 * (k[2] + t2 * k[3]))));
}

static double kb_dthd(const double *k, double th) {
    double t2 = th * th;
    return 1.0 + t2 * (3 * k[0] + t2 * (5 * k[1] + t2 * (7 * k[2] + t2 * 9 * k[3])));
}

/* Invert theta_d(theta) = r on [0, theta_lim] (monotone there): safeguarded Newton. */
static double kb_theta(const ocam *c, double r) {
    double lo = 0.0, hi = c->thlim;
    double th = r < hi ? r : hi;
    for (int it = 0; it < 200; ++it) {
        double f = kb_thd(c->k, th) - r;
        if (f > 0) hi = th; else lo = th;
        double fp = kb_dthd(c->k, th);
        double nt = (fp > 0) ? th - f / fp : 0.5 * (lo + hi);
        if (!(nt > lo && nt < hi)) nt = 0.5 * (lo + hi);
        if (fabs(nt - th) <= 1e-16 * (1.0 + th)) { th = nt; break; }
        th = nt;
        if (hi - lo < 1e-17) break;
    }
    return th;
}

/* Pi^-1: world direction (unit) of image point (x, y). */
static void unproject(const ocam *c, double x, double y, double d[3]) {
    double a = (x - c->cx) / c->fx, b = (y - c->cy) / c->fy, v[3];
    if (c->model == 0) {
        double n = sqrt(a * a + b * b + 1.0);
        v[0] = a / n; v[1] = b / n; v[2] = 1.0 / n;
    } else {
        double r = sqrt(a * a + b * b);
        double th = kb_theta(c, r);
        if (r > 0) {
            v[0] = sin(th) * a / r;
            v[1] = sin(th) * b / r;
        } else {
            v[0] = v[1] = 0.0;
        }
        v[2] = cos(th);
    }
    for (int i = 0; i < 3; ++i)
        d[i] = c->R[3 * i] * v[0] + c->R[3 * i + 1] * v[1] + c->R[3 * i + 2] * v[2];
}

/* Centre ray and the two half-pixel edge differentials delta_i = d_i - d
 * (backward difference when the forward edge point is outside the valid disc). */
static int pixel_rays(const ocam *c, double x, double y, double d[3], double dx[3], double dy[3]) {
    if (!f32_valid_xy(c, x, y)) return 0;
    double t[3];
    unproject(c, x, y, d);
    if (f32_valid_xy(c, x + 0.5, y)) {
        unproject(c, x + 0.5, y, t);
        for (int i = 0; i < 3; ++i) dx[i] = t[i] - d[i];
    } else {
        unproject(c, x - 0.5, y, t);
        for (int i = 0; i < 3; ++i) dx[i] = d[i] - t[i];
    }
    if (f32_valid_xy(c, x, y + 0.5)) {
        unproject(c, x, y + 0.5, t);
        for (int i = 0; i < 3; ++i) dy[i] = t[i] - d[i];
    } else {
        unproject(c, x, y - 0.5, t);
        for (int i = 0; i < 3; ++i) dy[i] = d[i] - t[i];
    }
    return 1;
}

/* Forward projection Pi (continuous pixel coordinates); returns 0 if the
 * point is not in front of / inside the camera's valid domain. */
static int project(const ocam *c, const double X[3], double *px, double *py) {
    double v[3], w[3];
    for (int i = 0; i < 3; ++i) w[i] = X[i] - c->o[i];
    for (int i = 0; i < 3; ++i) v[i] = c->Rinv[3 * i] * w[0] + c->Rinv[3 * i + 1] * w[1] + c->Rinv[3 * i + 2] * w[2];
    if (c->model == 0) {
        if (v[2] <= 0) return 0;
        *px = c->fx * v[0] / v[2] + c->cx;
        *py = c->fy * v[1] / v[2] + c->cy;
        return 1;
    }
    double rho = sqrt(v[0] * v[0] + v[1] * v[1]);
    double th = atan2(rho, v[2]);
    if (th > c->thlim) return 0;
    double td = kb_thd(c->k, th);
    if (rho > 0) {
        *px = c->fx * td * v[0] / rho + c->cx;
        *py = c->fy * td * v[1] / rho + c->cy;
    } else {
        *px = c->cx; *py = c->cy;
    }
    return 1;
}

/* ------------------------------------------------------------------ gaussians */

typedef struct {
    double mu[3], W[9], Winv[9], s[3], seff[3], sig, sig_eff, rho2, rgb[3], L;
    double key;  /* depth key: |mu - o| by the FP32 rule (see f32_depth_key) */
} ogauss;

/* The depth order is decided in FP32 (the same decision on every side):
 * key = sqrt((v0*v0 + v1*v1) + v2*v2), v = mu - o, each op one rounded FP32 op. */
static double f32_depth_key(const double *mu, const double *o) {
    float v0 = (float)mu[0] - (float)o[0], v1 = (float)mu[1] - (float)o[1], v2 = (float)mu[2] - (float)o[2];
    float L2 = (v0 * v0 + v1 * v1) + v2 * v2;
    return (double)sqrtf(L2);
}

/* Real spherical harmonics up to degree 3 (positive-constant real basis). */
static void sh_basis(const double v[3], double Y[16]) {
    const double PI = 3.14159265358979323846;
    double x = v[0], y = v[1], z = v[2];
    Y[0] = 0.5 * sqrt(1.0 / PI);
    double c1 = sqrt(3.0 / (4.0 * PI));
    Y[1] = c1 * y; Y[2] = c1 * z; Y[3] = c1 * x;
    double c2a = 0.5 * sqrt(15.0 / PI), c2b = 0.25 * sqrt(5.0 / PI), c2c = 0.25 * sqrt(15.0 / PI);
    Y[4] = c2a * x * y;
    Y[5] = c2a * y * z;
    Y[6] = c2b * (3.0 * z * z - 1.0);
    Y[7] = c2a * x * z;
    Y[8] = c2c * (x * x - y * y);
    double c3a = 0.25 * sqrt(35.0 / (2.0 * PI)), c3b = 0.5 * sqrt(105.0 / PI);
    double c3c = 0.25 * sqrt(21.0 / (2.0 * PI)), c3d = 0.25 * sqrt(7.0 / PI), c3e = 0.25 * sqrt(105.0 / PI);
    Y[9] = c3a * y * (3.0 * x * x - y * y);
    Y[10] = c3b * x * y * z;
    Y[11] = c3c * y * (5.0 * z * z - 1.0);
    Y[12] = c3d * z * (5.0 * z * z - 3.0);
    Y[13] = c3c * x * (5.0 * z * z - 1.0);
    Y[14] = c3e * z * (x * x - y * y);
    Y[15] = c3a * x * (x * x - 3.0 * y * y);
}

static void prep_gauss(const double o[3], const double *mu, const double *ls, const double *q,
                       double logit, const double *sh, int deg, double rho2, ogauss *g) {
    double qn = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
    double w = q[0] / qn, x = q[1] / qn, y = q[2] / qn, z = q[3] / qn;
    double R[9] = {1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y),
                   2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x),
                   2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)};
    g->rho2 = rho2;
    g->sig = 1.0 / (1.0 + exp(-logit));
    g->sig_eff = g->sig;
    for (int i = 0; i < 3; ++i) {
        g->mu[i] = mu[i];
        g->s[i] = exp(ls[i]);
        g->seff[i] = sqrt(g->s[i] * g->s[i] + rho2);  /* Eq. 10: s_i -> sqrt(s_i^2 + rho^2) */
        g->sig_eff *= g->s[i] / g->seff[i];
    }
    /* W = S_eff^-1 R^T ; W^-1 = R S_eff */
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            g->W[3 * i + j] = R[3 * j + i] / g->seff[i];
            g->Winv[3 * i + j] = R[3 * i + j] * g->seff[j];
        }
    double v[3];
    for (int i = 0; i < 3; ++i) v[i] = mu[i] - o[i];
    g->L = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
    g->key = f32_depth_key(mu, o);
    for (int i = 0; i < 3; ++i) v[i] /= g->L;
    double Y[16];
    sh_basis(v, Y);
    int K = (deg + 1) * (deg + 1);
    for (int c = 0; c < 3; ++c) {
        double acc = 0;
        for (int j = 0; j < K; ++j) acc += sh[3 * j + c] * Y[j];
        acc += 0.5;
        g->rgb[c] = acc > 0 ? acc : 0.0;
    }
}

/* The SH basis of n directions v[n*3] into Y[n*16] (exported so that the
 * tests can pin it against its definition). */
void or_sh_basis(int n, const double *v, double *Y) {
    for (int i = 0; i < n; ++i) sh_basis(v + 3 * (size_t)i, Y + 16 * (size_t)i);
}

/* ------------------------------------------------------------------ 3x3 helpers */

static void mv3(const double *M, const double *v, double *out) {
    for (int i = 0; i < 3; ++i) out[i] = M[3 * i] * v[0] + M[3 * i + 1] * v[1] + M[3 * i + 2] * v[2];
}

static double dot3(const double *a, const double *b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

static void mm3(const double *A, const double *B, double *C) {
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double s = 0;
            for (int k = 0; k < 3; ++k) s += A[3 * i + k] * B[3 * k + j];
            C[3 * i + j] = s;
        }
}

static void transpose3(const double *A, double *At) {
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) At[3 * j + i] = A[3 * i + j];
}

/* Cyclic Jacobi eigen-decomposition of a symmetric 3x3: A = V diag(lam) V^T. */
static void jacobi3(const double *Ain, double lam[3], double V[9]) {
    double A[9];
    memcpy(A, Ain, sizeof(A));
    for (int i = 0; i < 9; ++i) V[i] = (i % 4 == 0) ? 1.0 : 0.0;
    for (int sweep = 0; sweep < 64; ++sweep) {
        double off = A[1] * A[1] + A[2] * A[2] + A[5] * A[5];
        double scale = A[0] * A[0] + A[4] * A[4] + A[8] * A[8] + 2 * off;
        if (off <= 1e-34 * scale || off == 0.0) break;
        for (int p = 0; p < 2; ++p)
            for (int q = p + 1; q < 3; ++q) {
                double apq = A[3 * p + q];
                if (apq == 0.0) continue;
                double app = A[3 * p + p], aqq = A[3 * q + q];
                double theta = (aqq - app) / (2.0 * apq);
                double t = (theta >= 0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
                double cth = 1.0 / sqrt(t * t + 1.0), sth = t * cth;
                for (int k = 0; k < 3; ++k) { /* A <- J^T A J, columns p,q */
                    double akp = A[3 * k + p], akq = A[3 * k + q];
                    A[3 * k + p] = cth * akp - sth * akq;
                    A[3 * k + q] = sth * akp + cth * akq;
                }
                for (int k = 0; k < 3; ++k) { /* rows p,q */
                    double apk = A[3 * p + k], aqk = A[3 * q + k];
                    A[3 * p + k] = cth * apk - sth * aqk;
                    A[3 * q + k] = sth * apk + cth * aqk;
                }
                for (int k = 0; k < 3; ++k) {
                    double vkp = V[3 * k + p], vkq = V[3 * k + q];
                    V[3 * k + p] = cth * vkp - sth * vkq;
                    V[3 * k + q] = sth * vkp + cth * vkq;
                }
            }
    }
    lam[0] = A[0]; lam[1] = A[4]; lam[2] = A[8];
}

/* ------------------------------------------------------------------ one pair */

enum { FILTER_NONE = 0, FILTER_ANISO = 1, FILTER_ISO = 2, FILTER_ZF = 3 };

/* Isotropic footprint variants (the comparison axis of Sec. 5: the isotropic
 * reduction the paper defers to its absent appendix, and the paraxial z/f
 * sizing of VKRayGS reimplemented in the same framework).  Both keep Eq. 6-9
 * and only replace the pixel's two half-edge differentials by a b1, a b2, with
 * (b1, b2) an orthonormal basis of the plane across d: the world footprint at
 * the max-response point is then isotropic across the ray, t^2 a^2 / 3 per
 * axis (Eq. 8), and independent of the basis chosen.
 *   FILTER_ISO: a^2 = (|dx_perp|^2 + |dy_perp|^2) / 2, the half-trace of the
 *     true footprint (the isotropic reduction the paper uses in Eq. 11);
 *   FILTER_ZF:  a = |<d, z_cam>| / (2 f_x): per-axis variance z^2 / (12 f_x^2)
 *     at depth z along the optical axis z_cam (paraxial pixel size z / f). */
static void footprint_variant(const ocam *c, int filter, const double d[3], double dx[3], double dy[3]) {
    if (filter != FILTER_ISO && filter != FILTER_ZF) return;
    double a2;
    if (filter == FILTER_ISO) {
        double px[3], py[3], sx = dot3(d, dx), sy = dot3(d, dy);
        for (int i = 0; i < 3; ++i) { px[i] = dx[i] - sx * d[i]; py[i] = dy[i] - sy * d[i]; }
        a2 = 0.5 * (dot3(px, px) + dot3(py, py));
    } else {
        const double z = d[0] * c->R[2] + d[1] * c->R[5] + d[2] * c->R[8];
        a2 = z * z / (4.0 * c->fx * c->fx);
    }
    /* b1: the coordinate axis least aligned with d, made orthogonal to d */
    int k = 0;
    for (int i = 1; i < 3; ++i) if (fabs(d[i]) < fabs(d[k])) k = i;
    double b1[3] = {0, 0, 0}, b2[3];
    b1[k] = 1.0;
    const double s = dot3(b1, d);
    for (int i = 0; i < 3; ++i) b1[i] -= s * d[i];
    const double nb = sqrt(dot3(b1, b1));
    for (int i = 0; i < 3; ++i) b1[i] /= nb;
    b2[0] = d[1] * b1[2] - d[2] * b1[1];
    b2[1] = d[2] * b1[0] - d[0] * b1[2];
    b2[2] = d[0] * b1[1] - d[1] * b1[0];
    const double a = sqrt(a2);
    for (int i = 0; i < 3; ++i) { dx[i] = a * b1[i]; dy[i] = a * b2[i]; }
}
enum { COMP_MARGINAL = 0, COMP_ADDITIVE = 1 };

/* detail[] layout (when non-NULL, 64 doubles):
 * [0] T  [1] t*  [2..4] q  [5..7] d_u  [8..10] e_x  [11..13] e_y
 * [14..22] Sigma_fp^u  [23..31] Sigma_render^u  [32] det A  [33] q^T A^-1 q  [34] D^2 */
static int pair_response(const ogauss *g, const double o[3], const double d[3], const double dx[3],
                         const double dy[3], int filter, int comp, double *T, double *ts_out,
                         double *detail) {
    double ou[3], du[3], w[3];
    for (int i = 0; i < 3; ++i) w[i] = o[i] - g->mu[i];
    mv3(g->W, w, ou);                 /* o_u = W (o - mu) */
    mv3(g->W, d, du);                 /* d_u = W d */
    double n = dot3(du, du);
    double ts = -dot3(ou, du) / n;    /* Eq. 2 */
    *ts_out = ts;
    double Mp[9];                     /* M_perp = I - d_u d_u^T / n */
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) Mp[3 * i + j] = (i == j ? 1.0 : 0.0) - du[i] * du[j] / n;
    double q[3];
    mv3(Mp, ou, q);                   /* q = M_perp o_u */
    double D2 = dot3(q, q);
    double Sfp[9] = {0}, Sr[9] = {0}, ex[3] = {0}, ey[3] = {0}, detA = 1.0, Qf = D2;
    if (filter != FILTER_NONE) {
        double MW[9], t1[3];
        mm3(Mp, g->W, MW);
        mv3(MW, dx, t1);
        for (int i = 0; i < 3; ++i) ex[i] = ts * t1[i];   /* Eq. 6 */
        mv3(MW, dy, t1);
        for (int i = 0; i < 3; ++i) ey[i] = ts * t1[i];
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) Sfp[3 * i + j] = (ex[i] * ex[j] + ey[i] * ey[j]) / 3.0;  /* Eq. 8 */
        if (comp == COMP_MARGINAL) {
            /* Eq. 12: W [ W^-1 Sfp W^-T - rho^2 I ]_+ W^T */
            double WinvT[9], WT[9], t9[9], F[9], lam[3], V[9], P[9];
            transpose3(g->Winv, WinvT);
            transpose3(g->W, WT);
            mm3(g->Winv, Sfp, t9);
            mm3(t9, WinvT, F);
            for (int i = 0; i < 3; ++i) F[4 * i] -= g->rho2;
            jacobi3(F, lam, V);
            for (int i = 0; i < 3; ++i)
                for (int j = 0; j < 3; ++j) {
                    double s = 0;
                    for (int k = 0; k < 3; ++k) s += V[3 * i + k] * (lam[k] > 0 ? lam[k] : 0.0) * V[3 * j + k];
                    P[3 * i + j] = s;
                }
            mm3(g->W, P, t9);
            mm3(t9, WT, Sr);
        } else {
            memcpy(Sr, Sfp, sizeof(Sr));
        }
        /* Eq. 9: A = I + Sigma_render is symmetric with A >= I (Sigma_render is
         * PSD by the clamp of Eq. 12), so det A and q^T A^-1 q are taken from its
         * eigen-decomposition: det A = prod(1 + mu_i), q^T A^-1 q =
         * sum (v_i . q)^2 / (1 + mu_i), mu_i >= 0 the eigenvalues of Sigma_render.
         * (An LU of A loses its small pivots when Sigma_render is nearly rank one
         * and huge, as for a flat Gaussian whose whitened footprint reaches 1e10.) */
        double Ss[9], mu[3], V[9];
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) Ss[3 * i + j] = 0.5 * (Sr[3 * i + j] + Sr[3 * j + i]);
        jacobi3(Ss, mu, V);
        detA = 1.0;
        Qf = 0.0;
        for (int k = 0; k < 3; ++k) {
            const double a = 1.0 + (mu[k] > 0 ? mu[k] : 0.0);
            const double vq = V[k] * q[0] + V[3 + k] * q[1] + V[6 + k] * q[2];
            detA *= a;
            Qf += vq * vq / a;
        }
    }
    *T = g->sig_eff / sqrt(detA) * exp(-0.5 * Qf);   /* Eq. 9 (C = 1) */
    if (detail) {
        detail[0] = *T; detail[1] = ts;
        for (int i = 0; i < 3; ++i) {
            detail[2 + i] = q[i]; detail[5 + i] = du[i]; detail[8 + i] = ex[i]; detail[11 + i] = ey[i];
        }
        for (int i = 0; i < 9; ++i) { detail[14 + i] = Sfp[i]; detail[23 + i] = Sr[i]; }
        detail[32] = detA; detail[33] = Qf; detail[34] = D2;
        detail[49] = g->sig_eff;
    }
    return ts > T_NEAR;
}

/* ------------------------------------------------------------------ scene handle */

typedef struct {
    int n, deg;
    const double *means, *log_scales, *quats, *logits, *sh, *rho2;
} oscene;

static void prep_all(const ocam *c, const oscene *s, ogauss *g) {
    int K = (s->deg + 1) * (s->deg + 1);
#pragma omp parallel for schedule(static)
    for (int i = 0; i < s->n; ++i)
        prep_gauss(c->o, s->means + 3 * (size_t)i, s->log_scales + 3 * (size_t)i, s->quats + 4 * (size_t)i,
                   s->logits[i], s->sh + (size_t)3 * K * i, s->deg, s->rho2 ? s->rho2[i] : 0.0, &g[i]);
}

/* Oracle-side conservative cull (FP64, own derivation): a pair with
 * T >= 1/255 has q^T A^-1 q <= kappa^2 = 2 ln(255 sigma), so the
 * perpendicular distance from mu to the ray is at most
 * kappa sqrt(s_max^2 + t*^2 m), m = (|dx|^2+|dy|^2)/3, and
 * t* <= (L + kappa s_max) / (1 - kappa r1 sqrt(m)), r1 = (r + 1/r)/2 with
 * r = s_max/s_min: the world half-edges f_i = delta_i - c_i d (Eq. 6 mapped
 * back to world space) keep delta_i's part across d, and their part along d
 * is at most beta |delta_i|, beta = max_d |P_perp Sigma^-1 d| / d^T Sigma^-1 d
 * = (r - 1/r)/2 (the two extreme eigenvalues of Sigma^-1), so
 * |f_i| <= sqrt(1 + beta^2) |delta_i| = r1 |delta_i|. */
static int oracle_keep(const ogauss *g, const double o[3], const double d[3], double m) {
    double k2 = 2.0 * log(255.0 * g->sig);
    if (!(k2 > 0)) return 0;
    double kap = sqrt(k2);
    double smax = g->seff[0], smin = g->seff[0];
    for (int i = 1; i < 3; ++i) {
        smax = g->seff[i] > smax ? g->seff[i] : smax;
        smin = g->seff[i] < smin ? g->seff[i] : smin;
    }
    double r = smax / smin, r1 = 0.5 * (r + 1.0 / r), sm = sqrt(m), c = kap * r1 * sm, tb, rf;
    if (c < 0.5) {
        tb = (g->L + kap * smax) / (1.0 - c);
        rf = kap * sqrt(smax * smax + tb * tb * r1 * r1 * m);
    } else {
        rf = 255.0 * kap * smax;
        tb = g->L + rf;
    }
    if (g->L <= rf) return 1;
    double v[3];
    for (int i = 0; i < 3; ++i) v[i] = g->mu[i] - o[i];
    double along = dot3(v, d);
    if (along <= 0) return 0;
    double p2 = dot3(v, v) - along * along;
    double rp = kap * sqrt(smax * smax + tb * tb * m);
    return p2 <= rp * rp * (1.0 + 1e-9) + 1e-300;
}

typedef struct {
    double L, T, ts;
    int idx;
} cand;

static int cand_cmp(const void *a, const void *b) {
    const cand *x = (const cand *)a, *y = (const cand *)b;
    if (x->L < y->L) return -1;
    if (x->L > y->L) return 1;
    return x->idx - y->idx;
}

/* Per-ray order (the paper's "sorted by max-response depth t*_k", taken per
 * pixel): by the pair's own t*, ties by the canonical key, then index. */
static int cand_cmp_ts(const void *a, const void *b) {
    const cand *x = (const cand *)a, *y = (const cand *)b;
    if (x->ts < y->ts) return -1;
    if (x->ts > y->ts) return 1;
    return cand_cmp(a, b);
}

/* Composite order of or_render: 0 the canonical per-Gaussian key |mu - o|
 * (what the GPU path does), 1 the exact per-ray t* order. */
enum { ORDER_KEY = 0, ORDER_TSTAR = 1 };

/* Flag bits of the near-threshold protocol. */
enum { FL_ALPHA_MIN = 1, FL_ALPHA_MAX = 2, FL_STOP = 4, FL_KEY_TIE = 8, FL_TNEAR = 16, FL_UT_NEAR = 32 };

/* Composite one pixel's candidates (Eq. 4 with the 3DGS conventions). */
/* *nalpha (optional): the number of candidates with T >= 1/255, whether or not
 * the pixel reached them before its stop. */
static void composite(cand *cs, int nc, const ogauss *g, double eps, double eps_key, double rgb[3],
                      double *Tout, int *flags, int *ncontrib, int *used_idx, int max_used, int order,
                      int *nalpha) {
    qsort(cs, nc, sizeof(cand), order == ORDER_TSTAR ? cand_cmp_ts : cand_cmp);
    if (nalpha) {
        int na = 0;
        for (int k = 0; k < nc; ++k) na += cs[k].T >= ALPHA_MIN;
        *nalpha = na;
    }
    double Tacc = 1.0, C[3] = {0, 0, 0};
    int fl = 0, nu = 0, prev = -1;
    for (int k = 0; k < nc; ++k) {
        double T = cs[k].T;
        if (fabs(cs[k].ts - T_NEAR) <= eps * T_NEAR) fl |= FL_TNEAR;
        if (order == ORDER_TSTAR) {
            /* a near tie in t* between two pairs that may contribute: the order may
             * go either way in another precision */
            if (eps_key > 0 && T >= ALPHA_MIN * (1.0 - eps)) {
                if (prev >= 0 && fabs(cs[k].ts - cs[prev].ts) <= eps_key * fabs(cs[k].ts)) fl |= FL_KEY_TIE;
                prev = k;
            }
        } else if (eps_key > 0 && k > 0 && fabs(cs[k].L - cs[k - 1].L) <= eps_key * cs[k].L) {
            fl |= FL_KEY_TIE;
        }
        if (fabs(T - ALPHA_MIN) <= eps * ALPHA_MIN) fl |= FL_ALPHA_MIN;
        if (fabs(T - ALPHA_MAX) <= eps * ALPHA_MAX) fl |= FL_ALPHA_MAX;
        if (T < ALPHA_MIN) continue;
        double a = T < ALPHA_MAX ? T : ALPHA_MAX;
        double test = Tacc * (1.0 - a);
        if (fabs(test - T_STOP) <= eps * T_STOP) fl |= FL_STOP;
        if (test < T_STOP) break;
        const ogauss *gg = &g[cs[k].idx];
        for (int c = 0; c < 3; ++c) C[c] += gg->rgb[c] * a * Tacc;
        Tacc = test;
        if (used_idx && nu < max_used) used_idx[nu] = cs[k].idx;
        ++nu;
    }
    for (int c = 0; c < 3; ++c) rgb[c] = C[c];
    *Tout = Tacc;
    *flags = fl;
    *ncontrib = nu;
}

/* ------------------------------------------------------------------ exported API */

/* Rays for a list of image points: d, delta_x, delta_y (each [npts*3]) and the FP32 valid rule. */
void or_rays(const double *campk, int npts, const double *xs, const double *ys, double *d, double *dx,
             double *dy, int *valid) {
    ocam c;
    unpack_cam(campk, &c);
#pragma omp parallel for schedule(static)
    for (int i = 0; i < npts; ++i) {
        valid[i] = pixel_rays(&c, xs[i], ys[i], d + 3 * (size_t)i, dx + 3 * (size_t)i, dy + 3 * (size_t)i);
        if (!valid[i])
            for (int j = 0; j < 3; ++j) d[3 * i + j] = dx[3 * i + j] = dy[3 * i + j] = 0.0;
    }
}

/* Per-Gaussian derived quantities for one camera centre: [n*24]
 * W(9) Winv(9) sig_eff rgb(3) L rho2 */
void or_gauss(const double *campk, int n, const double *means, const double *log_scales, const double *quats,
              const double *logits, const double *sh, int deg, const double *rho2, double *out) {
    ocam c;
    unpack_cam(campk, &c);
    oscene s = {n, deg, means, log_scales, quats, logits, sh, rho2};
    ogauss *g = (ogauss *)malloc(sizeof(ogauss) * (size_t)(n > 0 ? n : 1));
    prep_all(&c, &s, g);
    for (int i = 0; i < n; ++i) {
        double *o = out + 24 * (size_t)i;
        memcpy(o, g[i].W, 9 * sizeof(double));
        memcpy(o + 9, g[i].Winv, 9 * sizeof(double));
        o[18] = g[i].sig_eff;
        o[19] = g[i].rgb[0]; o[20] = g[i].rgb[1]; o[21] = g[i].rgb[2];
        o[22] = g[i].L; o[23] = g[i].rho2;
    }
    free(g);
}

/* One pixel-Gaussian pair at image point (x, y), with all intermediate quantities. */
int or_pair_detail(const double *campk, double x, double y, const double *mu, const double *ls, const double *q,
                   double logit, double rho2, int filter, int comp, double *detail) {
    ocam c;
    unpack_cam(campk, &c);
    double d[3], dx[3], dy[3], sh[3] = {0, 0, 0}, ts, T;
    if (!pixel_rays(&c, x, y, d, dx, dy)) return -1;
    footprint_variant(&c, filter, d, dx, dy);
    ogauss g;
    prep_gauss(c.o, mu, ls, q, logit, sh, 0, rho2, &g);
    memset(detail, 0, 64 * sizeof(double));
    int ok = pair_response(&g, c.o, d, dx, dy, filter, comp, &T, &ts, detail);
    for (int i = 0; i < 3; ++i) { detail[40 + i] = d[i]; detail[43 + i] = dx[i]; detail[46 + i] = dy[i]; }
    return ok;
}

/* Pair response for explicit rays (d, delta_x, delta_y given), used by quadrature pins. */
double or_pair_rays(const double *o, const double *d, const double *dx, const double *dy, const double *mu,
                    const double *ls, const double *q, double logit, double rho2, int filter, int comp,
                    double *detail) {
    double sh[3] = {0, 0, 0}, ts, T;
    ogauss g;
    prep_gauss(o, mu, ls, q, logit, sh, 0, rho2, &g);
    if (detail) memset(detail, 0, 64 * sizeof(double));
    pair_response(&g, o, d, dx, dy, filter, comp, &T, &ts, detail);
    return T;
}

/* Supersampled pixel-bundle reference (Eq. 5 with the w = delta(t - t*) response,
 * C = 1): mean over nsub x nsub sub-pixel centres of sigma_eff exp(-D^2(xi)/2). */
double or_bundle(const double *campk, double x, double y, const double *mu, const double *ls, const double *q,
                 double logit, double rho2, int nsub) {
    ocam c;
    unpack_cam(campk, &c);
    double sh[3] = {0, 0, 0};
    ogauss g;
    prep_gauss(c.o, mu, ls, q, logit, sh, 0, rho2, &g);
    double acc = 0;
    int cnt = 0;
    for (int j = 0; j < nsub; ++j)
        for (int i = 0; i < nsub; ++i) {
            double xi = x - 0.5 + (i + 0.5) / nsub, yi = y - 0.5 + (j + 0.5) / nsub, d[3], ts, T;
            if (!f32_valid_xy(&c, xi, yi)) continue;
            unproject(&c, xi, yi, d);
            double z[3] = {0, 0, 0};
            pair_response(&g, c.o, d, z, z, FILTER_NONE, COMP_MARGINAL, &T, &ts, NULL);
            acc += T;
            ++cnt;
        }
    return cnt ? acc / cnt : 0.0;
}

/* Render a list of pixels (npix indices into the W x H grid; NULL = all).
 * Outputs rgb[npix*3], T[npix], flags[npix], ncontrib[npix]; optionally the
 * ids of the contributing Gaussians (used[npix*max_used]).  gate (optional,
 * from or_ut_gate): the pixel's tile must be kept for a Gaussian to be
 * evaluated; a contributing pair whose gate entry is ambiguous sets FL_UT_NEAR.
 * nalpha (optional, [npix]): per pixel, the pairs with T >= 1/255. */
void or_render(const double *campk, int n, const double *means, const double *log_scales, const double *quats,
               const double *logits, const double *sh, int deg, const double *rho2, int filter, int comp,
               int npix, const int *pix, int cull, double eps, double eps_key, double *rgb, double *Tout,
               int *flags, int *ncontrib, int *used, int max_used, int order, const unsigned char *gate,
               int *nalpha) {
    ocam c;
    unpack_cam(campk, &c);
    oscene s = {n, deg, means, log_scales, quats, logits, sh, rho2};
    ogauss *g = (ogauss *)malloc(sizeof(ogauss) * (size_t)(n > 0 ? n : 1));
    prep_all(&c, &s, g);
    int total = pix ? npix : c.W * c.H;
    const int ntx = (c.W + UT_TILE - 1) / UT_TILE, nt = ntx * ((c.H + UT_TILE - 1) / UT_TILE);
#pragma omp parallel
    {
        cand *cs = (cand *)malloc(sizeof(cand) * (size_t)(n > 0 ? n : 1));
#pragma omp for schedule(dynamic, 16)
        for (int t = 0; t < total; ++t) {
            int p = pix ? pix[t] : t;
            double x = (p % c.W) + 0.5, y = (p / c.W) + 0.5, d[3], dx[3], dy[3];
            double *o_rgb = rgb + 3 * (size_t)t;
            int *u = used ? used + (size_t)max_used * t : NULL;
            if (!pixel_rays(&c, x, y, d, dx, dy)) {
                o_rgb[0] = o_rgb[1] = o_rgb[2] = 0.0;
                Tout[t] = 1.0;
                flags[t] = 0;
                ncontrib[t] = 0;
                if (nalpha) nalpha[t] = 0;
                continue;
            }
            footprint_variant(&c, filter, d, dx, dy);
            double m = (dot3(dx, dx) + dot3(dy, dy)) / 3.0;
            int nc = 0, utnear = 0;
            const size_t tile = (size_t)((p / c.W) / UT_TILE) * ntx + (p % c.W) / UT_TILE;
            for (int k = 0; k < n; ++k) {
                /* UT binning: only the gate's tiles are evaluated (Sec. 3, 3DGUT backbone) */
                const int gv = gate ? gate[(size_t)k * nt + tile] : 1;
                if (gv == 0) continue;
                if (cull && !oracle_keep(&g[k], c.o, d, m)) continue;
                double T, ts;
                if (!pair_response(&g[k], c.o, d, dx, dy, filter, comp, &T, &ts, NULL)) {
                    if (fabs(ts - T_NEAR) <= eps * T_NEAR && T >= ALPHA_MIN * (1 - eps)) {
                        cs[nc].L = g[k].key; cs[nc].T = 0.0; cs[nc].ts = ts; cs[nc].idx = k; ++nc;
                    }
                    continue;
                }
                if (T < ALPHA_MIN * (1.0 - eps)) continue;
                if (gv == 2) utnear = 1;
                cs[nc].L = g[k].key; cs[nc].T = T; cs[nc].ts = ts; cs[nc].idx = k;
                ++nc;
            }
            composite(cs, nc, g, eps, eps_key, o_rgb, &Tout[t], &flags[t], &ncontrib[t], u, max_used, order,
                      nalpha ? &nalpha[t] : NULL);
            if (utnear) flags[t] |= FL_UT_NEAR;
        }
        free(cs);
    }
    free(g);
}

/* Dense sub-ray reference of a finite pixel (the multi-Gaussian counterpart of
 * or_bundle, Eq. 5): every pixel is split into nsub x nsub sub-pixels whose
 * centre rays are composited on their own (centre-ray responses, Eq. 3 with
 * C = 1, the compositing rules of Eq. 4, order by `order`), and the sub-ray
 * colours and transmittances are averaged over the valid sub-pixels. */
void or_render_subrays(const double *campk, int n, const double *means, const double *log_scales,
                       const double *quats, const double *logits, const double *sh, int deg, const double *rho2,
                       int npix, const int *pix, int nsub, int order, double *rgb, double *Tout) {
    ocam c;
    unpack_cam(campk, &c);
    oscene s = {n, deg, means, log_scales, quats, logits, sh, rho2};
    ogauss *g = (ogauss *)malloc(sizeof(ogauss) * (size_t)(n > 0 ? n : 1));
    prep_all(&c, &s, g);
    int total = pix ? npix : c.W * c.H;
#pragma omp parallel
    {
        cand *cs = (cand *)malloc(sizeof(cand) * (size_t)(n > 0 ? n : 1));
#pragma omp for schedule(dynamic, 4)
        for (int t = 0; t < total; ++t) {
            int p = pix ? pix[t] : t;
            double acc[3] = {0, 0, 0}, accT = 0;
            int cnt = 0;
            for (int j = 0; j < nsub; ++j)
                for (int i = 0; i < nsub; ++i) {
                    double x = (p % c.W) + (i + 0.5) / nsub, y = (p / c.W) + (j + 0.5) / nsub, d[3];
                    if (!f32_valid_xy(&c, x, y)) continue;
                    unproject(&c, x, y, d);
                    double z[3] = {0, 0, 0};
                    int nc = 0;
                    for (int k = 0; k < n; ++k) {
                        double T, ts;
                        if (!pair_response(&g[k], c.o, d, z, z, FILTER_NONE, COMP_MARGINAL, &T, &ts, NULL)) continue;
                        if (T < ALPHA_MIN) continue;
                        cs[nc].L = g[k].key; cs[nc].T = T; cs[nc].ts = ts; cs[nc].idx = k;
                        ++nc;
                    }
                    double sub_rgb[3], sub_T;
                    int fl, nu;
                    composite(cs, nc, g, 0.0, 0.0, sub_rgb, &sub_T, &fl, &nu, NULL, 0, order, NULL);
                    for (int q = 0; q < 3; ++q) acc[q] += sub_rgb[q];
                    accT += sub_T;
                    ++cnt;
                }
            for (int q = 0; q < 3; ++q) rgb[3 * (size_t)t + q] = cnt ? acc[q] / cnt : 0.0;
            Tout[t] = cnt ? accT / cnt : 1.0;
        }
        free(cs);
    }
    free(g);
}

/* All pixel-Gaussian pairs with T >= thr (for the binning-conservativeness check).
 * Returns the number of pairs found (writes at most cap of them as pix, gauss). */
long or_pairs_above(const double *campk, int n, const double *means, const double *log_scales,
                    const double *quats, const double *logits, const double *rho2, double thr, long cap,
                    int *out_pix, int *out_g) {
    ocam c;
    unpack_cam(campk, &c);
    double sh0[3] = {0, 0, 0};
    ogauss *g = (ogauss *)malloc(sizeof(ogauss) * (size_t)(n > 0 ? n : 1));
    for (int i = 0; i < n; ++i)
        prep_gauss(c.o, means + 3 * (size_t)i, log_scales + 3 * (size_t)i, quats + 4 * (size_t)i, logits[i], sh0,
                   0, rho2 ? rho2[i] : 0.0, &g[i]);
    int P = c.W * c.H;
    long *cnt = (long *)calloc((size_t)P + 1, sizeof(long));
    /* pass 1: count per pixel; pass 2: fill in pixel order */
    for (int pass = 0; pass < 2; ++pass) {
#pragma omp parallel for schedule(dynamic, 8)
        for (int p = 0; p < P; ++p) {
            double x = (p % c.W) + 0.5, y = (p / c.W) + 0.5, d[3], dx[3], dy[3];
            if (!pixel_rays(&c, x, y, d, dx, dy)) continue;
            long k0 = pass ? cnt[p] : 0, k = k0;
            for (int j = 0; j < n; ++j) {
                double T, ts;
                pair_response(&g[j], c.o, d, dx, dy, FILTER_ANISO, COMP_MARGINAL, &T, &ts, NULL);
                if (ts > T_NEAR * (1 - 1e-6) && T >= thr) {
                    if (pass && k < cap) { out_pix[k] = p; out_g[k] = j; }
                    ++k;
                }
            }
            if (!pass) cnt[p + 1] = k - k0;
        }
        if (!pass)
            for (int p = 0; p < P; ++p) cnt[p + 1] += cnt[p];
    }
    long total = cnt[P];
    free(cnt);
    free(g);
    return total;
}

/* Eq. 11: rho^2 = min over visible training views of tr(Sigma_fp)/2 at the
 * pixel onto which mu projects, evaluated before whitening (world space):
 * p = Pi_v(mu) (continuous), d = (mu - o)/|mu - o|, t = |mu - o|,
 * e_i = t (I - d d^T)(d_i - d), rho_v^2 = (|e_x|^2 + |e_y|^2)/6.
 * Visible: |mu - o| > 0.2 and Pi_v(mu) inside the image and the valid domain.
 * Never visible: rho^2 = 0.  cams: nv packed cameras. */
void or_floor(int nv, const double *cams, int n, const double *means, double *rho2) {
    ocam *cs = (ocam *)malloc(sizeof(ocam) * (size_t)(nv > 0 ? nv : 1));
    for (int v = 0; v < nv; ++v) unpack_cam(cams + 24 * (size_t)v, &cs[v]);
#pragma omp parallel for schedule(static)
    for (int i = 0; i < n; ++i) {
        double best = INFINITY;
        const double *mu = means + 3 * (size_t)i;
        for (int v = 0; v < nv; ++v) {
            const ocam *c = &cs[v];
            double w[3], px, py;
            for (int j = 0; j < 3; ++j) w[j] = mu[j] - c->o[j];
            double t = sqrt(dot3(w, w));
            if (!(t > 0.2)) continue;
            if (!project(c, mu, &px, &py)) continue;
            if (!(px >= 0 && px < c->W && py >= 0 && py < c->H)) continue;
            if (!f32_valid_xy(c, px, py)) continue;
            double d[3], e[3], tt[3], acc = 0;
            for (int j = 0; j < 3; ++j) d[j] = w[j] / t;
            for (int ax = 0; ax < 2; ++ax) {
                double xp = px + (ax == 0 ? 0.5 : 0.0), yp = py + (ax == 1 ? 0.5 : 0.0), sgn = 1.0;
                if (!f32_valid_xy(c, xp, yp)) {
                    xp = px - (ax == 0 ? 0.5 : 0.0);
                    yp = py - (ax == 1 ? 0.5 : 0.0);
                    sgn = -1.0;
                }
                unproject(c, xp, yp, tt);
                for (int j = 0; j < 3; ++j) e[j] = sgn * (tt[j] - d[j]);
                double along = dot3(e, d);
                for (int j = 0; j < 3; ++j) e[j] = t * (e[j] - along * d[j]);
                acc += dot3(e, e);
            }
            double r = acc / 6.0;
            if (r < best) best = r;
        }
        rho2[i] = isinf(best) ? 0.0 : best;
    }
    free(cs);
}

/* ------------------------------------------------------------------ unscented-transform binning
 *
 * The alternative binning backbone.  The paper plugs its response into two
 * backbones (Sec. 3): 3DGEER and 3DGUT, and 3DGUT bounds each Gaussian on the
 * image with an unscented transform (UT) of its 3D distribution through the
 * camera model instead of a Jacobian.  The response (Eq. 9) is unchanged; only
 * the set of (Gaussian, tile) pairs that is evaluated changes.  Definition
 * (the scaled UT of Julier and Uhlmann with alpha = 1, beta = 2, kappa = 0 in
 * n = 3 dimensions, so lambda = 0):
 *   sigma points  X_0 = mu, X_{+-i} = mu +- sqrt(3) s_eff,i R_i  (i = 1..3),
 *                 R_i the i-th principal axis, s_eff,i the floored scale (Eq. 10)
 *   weights       mean w_0 = 0, w_{+-i} = 1/6; covariance w_0 = 2, w_{+-i} = 1/6
 *   image         y_j = Pi(X_j) (the camera's own model), ybar = sum_j w_j y_j,
 *                 Sigma_2 = sum_j w^c_j (y_j - ybar)(y_j - ybar)^T + I/12
 *                 (1/12 px^2: the moment-matched variance of the half-pixel
 *                 parallelogram of Eq. 8, seen on the image)
 *   extent        k^2 = 2 ln(255 sigma_eff): alpha >= 1/255 needs a Mahalanobis
 *                 distance^2 of at most k^2
 *   tile test     keep tile (tx, ty) iff the minimum over its pixel-centre
 *                 rectangle [8 tx + 1/2, min(8 tx + 15/2, W - 1/2)] x (same in y)
 *                 of (y - ybar)^T Sigma_2^-1 (y - ybar) is at most k^2
 *   fallback      the Gaussian keeps the conservative angular-tile rule when
 *                 the rule's flag is not 1 (culled or pass-all), or when a
 *                 sigma point leaves the camera's domain: pinhole p_z < 0.1 |p|
 *                 (camera frame), fisheye polar angle > theta_lim.
 * FP64 decisions near a threshold are reported as ambiguous (gate value 2): an
 * FP32 implementation may take them either way (the ellipse test within a
 * relative eps of k^2, the domain test within a relative 1e-5 of its limit). */

#define UT_COSMIN 0.1
#define UT_VLP (1.0 / 12.0)
/* relative band of the domain decision reported as ambiguous: far above the
 * FP32 error of a camera-frame direction (~1e-7), far below the gate's eps */
#define UT_EPS_DOMAIN 1e-5

/* Minimum over [x0,x1] x [y0,y1] of Q(y) = (y - c)^T [[A,B],[B,C]] (y - c)
 * (A, C > 0, AC > B^2).  Q is convex, so when c lies outside the rectangle the
 * minimum is on its boundary; on an edge x = X it is at y = c_y - B (X - c_x) / C
 * clamped to the edge (and symmetrically on y = Y). */
double or_ut_rect_min(double cx, double cy, double A, double B, double C, double x0, double x1, double y0,
                      double y1) {
    const double dx0 = x0 - cx, dx1 = x1 - cx, dy0 = y0 - cy, dy1 = y1 - cy;
    if (dx0 <= 0 && dx1 >= 0 && dy0 <= 0 && dy1 >= 0) return 0.0;
    const double ex[2] = {dx0, dx1}, ey[2] = {dy0, dy1};
    double best = INFINITY;
    for (int e = 0; e < 2; ++e) {
        double x = ex[e], y = -B * x / C;
        y = y < dy0 ? dy0 : (y > dy1 ? dy1 : y);
        double q = A * x * x + 2.0 * B * x * y + C * y * y;
        if (q < best) best = q;
        y = ey[e];
        x = -B * y / A;
        x = x < dx0 ? dx0 : (x > dx1 ? dx1 : x);
        q = A * x * x + 2.0 * B * x * y + C * y * y;
        if (q < best) best = q;
    }
    return best;
}

/* UT image ellipse of one Gaussian: returns 1 with ybar[2], conic[3] =
 * Sigma_2^-1 (A, B, C) and k^2; 0 when a sigma point is outside the camera's
 * domain.  *amb = 1 when that domain decision lies within UT_EPS_DOMAIN of its limit. */
static int ut_project(const ocam *c, const ogauss *g, double ybar[2], double conic[3], double *k2, int *amb) {
    double X[7][3], y[7][2];
    const double r3 = sqrt(3.0);
    for (int k = 0; k < 3; ++k) X[0][k] = g->mu[k];
    for (int i = 0; i < 3; ++i)
        for (int k = 0; k < 3; ++k) {
            /* column i of W^-1 = R S_eff is s_eff,i R_i */
            X[1 + 2 * i][k] = g->mu[k] + r3 * g->Winv[3 * k + i];
            X[2 + 2 * i][k] = g->mu[k] - r3 * g->Winv[3 * k + i];
        }
    int ok = 1;
    *amb = 0;
    for (int j = 0; j < 7; ++j) {
        double w[3], p[3];
        for (int k = 0; k < 3; ++k) w[k] = X[j][k] - c->o[k];
        mv3(c->Rinv, w, p);
        if (c->model == 0) {
            const double nrm = sqrt(dot3(p, p));
            const double cs = nrm > 0 ? p[2] / nrm : -1.0;
            if (fabs(cs - UT_COSMIN) <= UT_EPS_DOMAIN * UT_COSMIN) *amb = 1;
            if (!(cs >= UT_COSMIN)) ok = 0;
        } else {
            const double th = atan2(sqrt(p[0] * p[0] + p[1] * p[1]), p[2]);
            if (fabs(th - c->thlim) <= UT_EPS_DOMAIN * c->thlim) *amb = 1;
            if (!(th <= c->thlim)) ok = 0;
        }
    }
    if (!ok) return 0;
    for (int j = 0; j < 7; ++j)
        if (!project(c, X[j], &y[j][0], &y[j][1])) return 0;
    double wm[7], wc[7];
    wm[0] = 0.0;
    wc[0] = 2.0;
    for (int j = 1; j < 7; ++j) wm[j] = wc[j] = 1.0 / 6.0;
    ybar[0] = ybar[1] = 0.0;
    for (int j = 0; j < 7; ++j) {
        ybar[0] += wm[j] * y[j][0];
        ybar[1] += wm[j] * y[j][1];
    }
    double Sxx = UT_VLP, Sxy = 0.0, Syy = UT_VLP;
    for (int j = 0; j < 7; ++j) {
        const double ax = y[j][0] - ybar[0], ay = y[j][1] - ybar[1];
        Sxx += wc[j] * ax * ax;
        Sxy += wc[j] * ax * ay;
        Syy += wc[j] * ay * ay;
    }
    const double det = Sxx * Syy - Sxy * Sxy;
    conic[0] = Syy / det;
    conic[1] = -Sxy / det;
    conic[2] = Sxx / det;
    *k2 = 2.0 * log(255.0 * g->sig_eff);
    return 1;
}

/* UT gate of every (Gaussian, tile), row-major tiles of 8 x 8 pixels:
 *   gate[n * ntiles]: 0 drop, 1 keep, 2 ambiguous (within eps of k^2);
 *   status[n]: 0 the angular-tile rule decides (flag != 1 or a sigma point
 *     outside the domain; its row of gate is all 1: that rule is conservative),
 *     1 UT, 2 the domain decision is ambiguous (row all 2);
 *   geo[n * 6] (optional): ybar (2), conic A B C, k^2 of status-1 Gaussians.
 * flags[n]: the angular-tile rule's per-Gaussian flag (0 culled, 1 normal, 2 pass-all). */
void or_ut_gate(const double *campk, int n, const double *means, const double *log_scales, const double *quats,
                const double *logits, const double *rho2, const int *flags, double eps, unsigned char *gate,
                int *status, double *geo) {
    ocam c;
    unpack_cam(campk, &c);
    const int ntx = (c.W + UT_TILE - 1) / UT_TILE, nty = (c.H + UT_TILE - 1) / UT_TILE, nt = ntx * nty;
    double *sh0 = (double *)calloc((size_t)3 * (n > 0 ? n : 1), sizeof(double));
#pragma omp parallel for schedule(dynamic, 16)
    for (int i = 0; i < n; ++i) {
        unsigned char *row = gate + (size_t)i * nt;
        double *gg = geo ? geo + 6 * (size_t)i : NULL;
        if (gg)
            for (int k = 0; k < 6; ++k) gg[k] = 0.0;
        if (flags[i] != 1) {
            status[i] = 0;
            memset(row, 1, (size_t)nt);
            continue;
        }
        ogauss g;
        prep_gauss(c.o, means + 3 * (size_t)i, log_scales + 3 * (size_t)i, quats + 4 * (size_t)i, logits[i],
                   sh0 + 3 * (size_t)i, 0, rho2 ? rho2[i] : 0.0, &g);
        double yb[2], cn[3], k2;
        int amb;
        const int ok = ut_project(&c, &g, yb, cn, &k2, &amb);
        if (amb) {
            status[i] = 2;
            memset(row, 2, (size_t)nt);
            continue;
        }
        if (!ok) {
            status[i] = 0;
            memset(row, 1, (size_t)nt);
            continue;
        }
        status[i] = 1;
        if (gg) {
            gg[0] = yb[0]; gg[1] = yb[1]; gg[2] = cn[0]; gg[3] = cn[1]; gg[4] = cn[2]; gg[5] = k2;
        }
        const double tol = eps * (k2 > 1.0 ? k2 : 1.0);
        for (int t = 0; t < nt; ++t) {
            const int tx = t % ntx, ty = t / ntx;
            const double x0 = UT_TILE * tx + 0.5, y0 = UT_TILE * ty + 0.5;
            double x1 = UT_TILE * tx + UT_TILE - 0.5, y1 = UT_TILE * ty + UT_TILE - 0.5;
            if (x1 > c.W - 0.5) x1 = c.W - 0.5;
            if (y1 > c.H - 0.5) y1 = c.H - 0.5;
            const double q = or_ut_rect_min(yb[0], yb[1], cn[0], cn[1], cn[2], x0, x1, y0, y1);
            row[t] = fabs(q - k2) <= tol ? 2 : (q <= k2 ? 1 : 0);
        }
    }
    free(sh0);
}

/* ======================================================================
 * FP32 emulation of the conservative angular-tile binning rule.
 *
 * Every line below is one correctly rounded FP32 operation (+, -, *, /,
 * sqrt, min, max, floor), evaluated in the order written; this file is
 * compiled with -ffp-contract=off.  The transcendental functions the rule
 * needs (exp for the scales, sin/cos for the KB direction) are replaced by
 * fixed polynomial evaluations written from their Taylor series, so the
 * same operation sequence gives the same bits everywhere.
 * ====================================================================== */

typedef struct {
    int model, W, H;
    float fx, fy, cx, cy, k[4], R[9], o[3], thlim, rlim2;
} fcam;

static void unpack_fcam(const double *p, fcam *c) {
    c->model = (int)p[0];
    c->W = (int)p[1];
    c->H = (int)p[2];
    c->fx = (float)p[3]; c->fy = (float)p[4]; c->cx = (float)p[5]; c->cy = (float)p[6];
    for (int i = 0; i < 4; ++i) c->k[i] = (float)p[7 + i];
    for (int i = 0; i < 9; ++i) c->R[i] = (float)p[11 + i];
    for (int i = 0; i < 3; ++i) c->o[i] = (float)p[20 + i];
    c->thlim = (float)p[23];
    float t2 = c->thlim * c->thlim;
    float pp = ((c->k[3] * t2 + c->k[2]) * t2 + c->k[1]) * t2 + c->k[0];
    float rl = c->thlim * (1.0f + t2 * pp);
    c->rlim2 = rl * rl;
}

static int fvalid(const fcam *c, float x, float y) {
    if (c->model == 0) return 1;
    float a = (x - c->cx) / c->fx;
    float b = (y - c->cy) / c->fy;
    float r2 = a * a + b * b;
    return r2 <= c->rlim2;
}

/* sin and cos on [0, 1.7] from their Taylor series (Horner, to x^17 / x^16). */
static void f_sincos(float t, float *sn, float *cs) {
    const float S1 = (float)(-1.0 / 6.0), S2 = (float)(1.0 / 120.0), S3 = (float)(-1.0 / 5040.0),
                S4 = (float)(1.0 / 362880.0), S5 = (float)(-1.0 / 39916800.0),
                S6 = (float)(1.0 / 6227020800.0), S7 = (float)(-1.0 / 1307674368000.0),
                S8 = (float)(1.0 / 355687428096000.0);
    const float C1 = (float)(-1.0 / 2.0), C2 = (float)(1.0 / 24.0), C3 = (float)(-1.0 / 720.0),
                C4 = (float)(1.0 / 40320.0), C5 = (float)(-1.0 / 3628800.0), C6 = (float)(1.0 / 479001600.0),
                C7 = (float)(-1.0 / 87178291200.0), C8 = (float)(1.0 / 20922789888000.0);
    float t2 = t * t;
    float s = S8;
    s = s * t2 + S7; s = s * t2 + S6; s = s * t2 + S5; s = s * t2 + S4;
    s = s * t2 + S3; s = s * t2 + S2; s = s * t2 + S1; s = s * t2 + 1.0f;
    *sn = s * t;
    float c = C8;
    c = c * t2 + C7; c = c * t2 + C6; c = c * t2 + C5; c = c * t2 + C4;
    c = c * t2 + C3; c = c * t2 + C2; c = c * t2 + C1; c = c * t2 + 1.0f;
    *cs = c;
}

/* FP32 ray direction of image point (x, y), world frame. */
static void fdir(const fcam *c, float x, float y, float out[3]) {
    float a = (x - c->cx) / c->fx;
    float b = (y - c->cy) / c->fy;
    float v0, v1, v2;
    if (c->model == 0) {
        float n2 = (a * a + b * b) + 1.0f;
        float s = sqrtf(n2);
        v0 = a / s; v1 = b / s; v2 = 1.0f / s;
    } else {
        float r2 = a * a + b * b;
        float r = sqrtf(r2);
        float th = fminf(r, c->thlim);
        for (int it = 0; it < 12; ++it) {
            float t2 = th * th;
            float p = ((c->k[3] * t2 + c->k[2]) * t2 + c->k[1]) * t2 + c->k[0];
            float f = th * (1.0f + t2 * p) - r;
            float dp = ((9.0f * c->k[3] * t2 + 7.0f * c->k[2]) * t2 + 5.0f * c->k[1]) * t2 + 3.0f * c->k[0];
            float fp = 1.0f + t2 * dp;
            th = th - f / fp;
            th = fminf(fmaxf(th, 0.0f), c->thlim);
        }
        float sn, cs;
        f_sincos(th, &sn, &cs);
        if (r > 0.0f) { v0 = (sn * a) / r; v1 = (sn * b) / r; }
        else { v0 = 0.0f; v1 = 0.0f; }
        v2 = cs;
    }
    for (int i = 0; i < 3; ++i) out[i] = (c->R[3 * i] * v0 + c->R[3 * i + 1] * v1) + c->R[3 * i + 2] * v2;
}

/* FP32 edge differential along one axis with the backward-difference rule. */
static void fedge(const fcam *c, float x, float y, const float d[3], int axis, float e[3]) {
    float xp = axis == 0 ? x + 0.5f : x, yp = axis == 1 ? y + 0.5f : y, t[3];
    if (fvalid(c, xp, yp)) {
        fdir(c, xp, yp, t);
        for (int i = 0; i < 3; ++i) e[i] = t[i] - d[i];
    } else {
        float xm = axis == 0 ? x - 0.5f : x, ym = axis == 1 ? y - 0.5f : y;
        fdir(c, xm, ym, t);
        for (int i = 0; i < 3; ++i) e[i] = d[i] - t[i];
    }
}

#define TILE 8

/* Tile cone table: per tile (row-major over ceil(W/8) x ceil(H/8)) 6 floats
 * a0 a1 a2 (axis = ray of the tile centre), sg = sin(gamma/2) (inflated),
 * cg = cos(gamma/2), m = max over pixels of (|dx|^2+|dy|^2)/3 (x1.01);
 * sg = -1 marks a tile without valid pixels. */
void or_tile_table(const double *campk, float *table) {
    fcam c;
    unpack_fcam(campk, &c);
    int tx_n = (c.W + TILE - 1) / TILE, ty_n = (c.H + TILE - 1) / TILE;
#pragma omp parallel for schedule(dynamic, 4)
    for (int t = 0; t < tx_n * ty_n; ++t) {
        int tx = t % tx_n, ty = t / tx_n;
        float a[3], d[3], ex[3], ey[3];
        fdir(&c, (float)(TILE * tx + TILE / 2), (float)(TILE * ty + TILE / 2), a);
        float ch2max = -1.0f, mmax = 0.0f;
        for (int j = TILE * ty; j < TILE * ty + TILE && j < c.H; ++j)
            for (int i = TILE * tx; i < TILE * tx + TILE && i < c.W; ++i) {
                float x = (float)i + 0.5f, y = (float)j + 0.5f;
                if (!fvalid(&c, x, y)) continue;
                fdir(&c, x, y, d);
                float e0 = a[0] - d[0], e1 = a[1] - d[1], e2 = a[2] - d[2];
                float ch2 = (e0 * e0 + e1 * e1) + e2 * e2;
                ch2max = fmaxf(ch2max, ch2);
                fedge(&c, x, y, d, 0, ex);
                fedge(&c, x, y, d, 1, ey);
                float mm = (((ex[0] * ex[0] + ex[1] * ex[1]) + ex[2] * ex[2]) +
                            ((ey[0] * ey[0] + ey[1] * ey[1]) + ey[2] * ey[2])) / 3.0f;
                mmax = fmaxf(mmax, mm);
            }
        float *o = table + 6 * (size_t)t;
        o[0] = a[0]; o[1] = a[1]; o[2] = a[2];
        if (ch2max < 0.0f) {
            o[3] = -1.0f; o[4] = 0.0f; o[5] = 0.0f;
            continue;
        }
        float sg = sqrtf(ch2max) * 0.5f + 2e-6f;
        sg = fminf(sg, 1.0f);
        o[3] = sg;
        o[4] = sqrtf(1.0f - sg * sg);
        o[5] = mmax * 1.01f;
    }
}

/* exp(x) from 2^k * sum_{j<=9} f^j/j!, x = k ln2 + f; |rel err| < 1e-5 on [-80,80]. */
static float f_exp(float x) {
    const float INV_LN2 = (float)(1.0 / 0.69314718055994530942), LN2F = (float)0.69314718055994530942;
    const float E2 = (float)(1.0 / 2.0), E3 = (float)(1.0 / 6.0), E4 = (float)(1.0 / 24.0),
                E5 = (float)(1.0 / 120.0), E6 = (float)(1.0 / 720.0), E7 = (float)(1.0 / 5040.0),
                E8 = (float)(1.0 / 40320.0), E9 = (float)(1.0 / 362880.0);
    x = fminf(fmaxf(x, -80.0f), 80.0f);
    float kf = floorf(x * INV_LN2);
    float f = x - kf * LN2F;
    float p = E9;
    p = p * f + E8; p = p * f + E7; p = p * f + E6; p = p * f + E5;
    p = p * f + E4; p = p * f + E3; p = p * f + E2; p = p * f + 1.0f; p = p * f + 1.0f;
    int k = (int)kf;
    union { uint32_t u; float f; } two;
    two.u = (uint32_t)(k + 127) << 23;
    return p * two.f;
}

/* Per-Gaussian binning record (16 floats): u0 u1 u2 L kap ks kr r1sq s2 flag
 * Sigma_eff (xx xy xz yy yz zz); flag: 0 culled (can never reach alpha >=
 * 1/255), 1 normal, 2 pass-all. */
static void fsigma(const float *q, const float *ls, float rho2, float *S);

static void fgauss(const fcam *c, const float *mu, const float *ls, const float *q, float logit, float rho2,
                   float *rec) {
    const float K255 = 11.082528f; /* >= 2 ln 255 */
    const float LN2LO = 0.6931471f; /* <= ln 2 */
    float lmax = fmaxf(fmaxf(ls[0], ls[1]), ls[2]);
    float lmin = fminf(fminf(ls[0], ls[1]), ls[2]);
    float s2 = f_exp(2.0f * lmax) * 1.0001f + rho2;
    float s2mn = f_exp(2.0f * lmin) * 0.9999f + rho2;
    float kap2 = K255 - 2.0f * fmaxf(fmaxf(0.0f, -logit), LN2LO - 0.5f * logit);
    float v0 = mu[0] - c->o[0], v1 = mu[1] - c->o[1], v2 = mu[2] - c->o[2];
    float L2 = (v0 * v0 + v1 * v1) + v2 * v2;
    float L = sqrtf(L2);
    for (int i = 0; i < 10; ++i) rec[i] = 0.0f;
    fsigma(q, ls, rho2, rec + 10);
    rec[3] = L;
    if (!(kap2 > 0.0f)) { rec[9] = 0.0f; return; }
    if (!(L > 0.0f)) { rec[9] = 2.0f; return; }
    rec[0] = v0 / L; rec[1] = v1 / L; rec[2] = v2 / L;
    float kap = sqrtf(kap2);
    float s = sqrtf(s2);
    float rr = s / sqrtf(s2mn);
    float r1 = fmaxf(((rr + 1.0f / rr) * 0.5f) * 1.00001f, 1.0f);
    rec[4] = kap;
    rec[5] = kap * s;
    rec[6] = kap * r1;
    rec[7] = r1 * r1;
    rec[8] = s2;
    rec[9] = 1.0f;
}

/* The per (Gaussian, tile) conservative test. */
static int ftest(const float *g, const float *t) {
    if (t[3] < 0.0f) return 0;
    if (g[9] == 0.0f) return 0;
    if (g[9] == 2.0f) return 1;
    float L = g[3], kap = g[4], ks = g[5], kr = g[6], r1sq = g[7], s2 = g[8];
    float m = t[5];
    float sm = sqrtf(m);
    float c = kr * sm;
    /* two valid bounds on |x* - mu| and t*, combined by min (monotone in m) */
    float rfc = 255.0f * ks;
    float tb, rf;
    if (c < 1.0f) {
        float tbf = (L + ks) / (1.0f - c);
        float rff = kap * sqrtf(s2 + ((tbf * tbf) * r1sq) * m);
        rf = fminf(rff, rfc);
        tb = fminf(tbf, L + rf);
    } else {
        rf = rfc;
        tb = L + rf;
    }
    if (L <= rf) return 1;
    float rp = kap * sqrtf(s2 + (tb * tb) * m);
    if (rp >= L) return 1;
    float sb = rp / L;
    float cb = sqrtf(1.0f - sb * sb);
    float sh2 = (sb * sb) / (2.0f * (1.0f + cb));
    float sbh = sqrtf(sh2);
    float cbh = sqrtf(1.0f - sh2);
    float sphi = sbh * t[4] + cbh * t[3];
    float e0 = g[0] - t[0], e1 = g[1] - t[1], e2 = g[2] - t[2];
    float ch2 = (e0 * e0 + e1 * e1) + e2 * e2;
    float lim = (2.0f * sphi) * 1.0001f + 4e-6f;
    return ch2 <= lim * lim;
}

/* Silhouette ellipse of the rule's bounding ellipsoid (pinhole cameras).
 * A contributing pair's ray meets E = {x : (x - mu)^T C^-1 (x - mu) <= kap^2},
 * C = Sigma_eff + t_b^2 m I; the lines through the camera centre that meet E
 * trace an ellipse on the image plane.  Scene part: Sigma_eff (xx xy xz yy yz
 * zz) from the FP32 quaternion and the rule's exp, s_eff^2 = exp(2 log s)
 * 1.0001 + rho^2. */
static void fsigma(const float *q, const float *ls, float rho2, float *S) {
    float n2 = ((q[0] * q[0] + q[1] * q[1]) + q[2] * q[2]) + q[3] * q[3];
    float inv = 1.0f / sqrtf(n2);
    float w = q[0] * inv, x = q[1] * inv, y = q[2] * inv, z = q[3] * inv;
    float R[9];
    R[0] = 1.0f - 2.0f * (y * y + z * z);
    R[1] = 2.0f * (x * y - w * z);
    R[2] = 2.0f * (x * z + w * y);
    R[3] = 2.0f * (x * y + w * z);
    R[4] = 1.0f - 2.0f * (x * x + z * z);
    R[5] = 2.0f * (y * z - w * x);
    R[6] = 2.0f * (x * z - w * y);
    R[7] = 2.0f * (y * z + w * x);
    R[8] = 1.0f - 2.0f * (x * x + y * y);
    float s2[3];
    for (int a = 0; a < 3; ++a) s2[a] = f_exp(2.0f * ls[a]) * 1.0001f + rho2;
    const int I[6] = {0, 0, 0, 1, 1, 2}, J[6] = {0, 1, 2, 1, 2, 2};
    for (int k = 0; k < 6; ++k) {
        int i = I[k], j = J[k];
        S[k] = ((R[3 * i] * R[3 * j]) * s2[0] + (R[3 * i + 1] * R[3 * j + 1]) * s2[1]) +
               (R[3 * i + 2] * R[3 * j + 2]) * s2[2];
    }
}

/* View part.  With v = (mu - o)/L in a frame F, C normalised by its mean
 * eigenvalue tau (+ 1e-4 I) and k^2 = kap^2 tau / L^2, a line of direction
 * d = (x, y, 1) (in F) meets E iff delta = d - v/v_z satisfies
 *   delta^T G delta - 2 h^T delta <= k0,  G = (a - k^2) Ci_xy - w_xy w_xy^T,
 *   h = k^2 w_xy / v_z, k0 = k^2 a / v_z^2, w = Ci v, a = v^T w.
 * Pinhole: F = the camera axes, the ellipse in pixels, el = (c_x, c_y, A, B, C,
 * 1.01 rhs, -B/C, -B/A).  Fisheye: F = (e1, e2, u), u = (mu - o)/L, e1 from the
 * world axis least aligned with u, so v = (0, 0, 1) and (x, y) are gnomonic
 * coordinates around u; el = (c_x, c_y, G00, G01, G11, sqrt(1.01 rhs), sqrt(tr G), e1).
 * Returns 0 when the test does not apply. */
static int fellipse(const fcam *c, const float *g, const float *mu, float m, float *el) {
    float L = g[3], kap = g[4], ks = g[5], kr = g[6], r1sq = g[7], s2 = g[8];
    const float *S = g + 10;
    float sm = sqrtf(m);
    float cc = kr * sm;
    float rfc = 255.0f * ks;
    float tb, rf;
    if (cc < 1.0f) {
        float tbf = (L + ks) / (1.0f - cc);
        float rff = kap * sqrtf(s2 + ((tbf * tbf) * r1sq) * m);
        rf = fminf(rff, rfc);
        tb = fminf(tbf, L + rf);
    } else {
        rf = rfc;
        tb = L + rf;
    }
    if (!(L > rf)) return 0;
    float w0 = mu[0] - c->o[0], w1 = mu[1] - c->o[1], w2 = mu[2] - c->o[2];
    float F[9], v[3];
    if (c->model == 0) {
        for (int k = 0; k < 9; ++k) F[k] = c->R[k];
        float iL = 1.0f / L;
        for (int j = 0; j < 3; ++j) v[j] = ((c->R[j] * w0 + c->R[3 + j] * w1) + c->R[6 + j] * w2) * iL;
        if (!(v[2] > 0.0f && v[2] * v[2] >= 0.05f)) return 0;
    } else {
        float u[3] = {w0 / L, w1 / L, w2 / L};
        float au0 = fabsf(u[0]), au1 = fabsf(u[1]), au2 = fabsf(u[2]);
        int k = (au0 <= au1 && au0 <= au2) ? 0 : (au1 <= au2 ? 1 : 2);
        float b[3] = {0.0f, 0.0f, 0.0f};
        b[k] = 1.0f;
        float uk = u[k];
        for (int j = 0; j < 3; ++j) b[j] = b[j] - uk * u[j];
        float nb = sqrtf((b[0] * b[0] + b[1] * b[1]) + b[2] * b[2]);
        float e1[3] = {b[0] / nb, b[1] / nb, b[2] / nb};
        float e2[3] = {u[1] * e1[2] - u[2] * e1[1], u[2] * e1[0] - u[0] * e1[2], u[0] * e1[1] - u[1] * e1[0]};
        for (int j = 0; j < 3; ++j) {
            F[3 * j] = e1[j];
            F[3 * j + 1] = e2[j];
            F[3 * j + 2] = u[j];
        }
        v[0] = 0.0f;
        v[1] = 0.0f;
        v[2] = 1.0f;
        el[7] = e1[0];
        el[8] = e1[1];
        el[9] = e1[2];
    }
    float Sf[9] = {S[0], S[1], S[2], S[1], S[3], S[4], S[2], S[4], S[5]};
    float T[9];
    for (int i = 0; i < 3; ++i)
        for (int k = 0; k < 3; ++k) T[3 * i + k] = (Sf[3 * i] * F[k] + Sf[3 * i + 1] * F[3 + k]) + Sf[3 * i + 2] * F[6 + k];
    float Cc[6];
    {
        const int I[6] = {0, 0, 0, 1, 1, 2}, J[6] = {0, 1, 2, 1, 2, 2};
        for (int k = 0; k < 6; ++k) {
            int j = I[k], l = J[k];
            Cc[k] = (F[j] * T[l] + F[3 + j] * T[3 + l]) + F[6 + j] * T[6 + l];
        }
    }
    float iso = (tb * tb) * m + 1e-5f * s2;
    Cc[0] = Cc[0] + iso;
    Cc[3] = Cc[3] + iso;
    Cc[5] = Cc[5] + iso;
    float tau = ((Cc[0] + Cc[3]) + Cc[5]) / 3.0f;
    float it = 1.0f / tau;
    float cxx = Cc[0] * it + 1e-4f, cxy = Cc[1] * it, cxz = Cc[2] * it;
    float cyy = Cc[3] * it + 1e-4f, cyz = Cc[4] * it, czz = Cc[5] * it + 1e-4f;
    float k2 = ((kap * kap) * tau) / (L * L);
    float a00 = cyy * czz - cyz * cyz;
    float a01 = cxz * cyz - cxy * czz;
    float a02 = cxy * cyz - cxz * cyy;
    float a11 = cxx * czz - cxz * cxz;
    float a12 = cxy * cxz - cxx * cyz;
    float det = (cxx * a00 + cxy * a01) + cxz * a02;
    if (!(det > 1e-12f)) return 0;
    float id = 1.0f / det;
    float i00 = a00 * id, i01 = a01 * id, i02 = a02 * id, i11 = a11 * id, i12 = a12 * id;
    float i22 = (cxx * cyy - cxy * cxy) * id;
    float wx = (i00 * v[0] + i01 * v[1]) + i02 * v[2];
    float wy = (i01 * v[0] + i11 * v[1]) + i12 * v[2];
    float wz = (i02 * v[0] + i12 * v[1]) + i22 * v[2];
    float a = (v[0] * wx + v[1] * wy) + v[2] * wz;
    float am = a - k2;
    if (!(am > 0.01f * k2)) return 0;
    float G00 = am * i00 - wx * wx;
    float G01 = am * i01 - wx * wy;
    float G11 = am * i11 - wy * wy;
    float dG = G00 * G11 - G01 * G01;
    float tG = G00 + G11;
    if (!(G00 > 0.0f && dG > 1e-6f * (tG * tG))) return 0;
    float ivz = 1.0f / v[2];
    float hx = (k2 * wx) * ivz, hy = (k2 * wy) * ivz;
    float k0 = (k2 * a) * (ivz * ivz);
    float idG = 1.0f / dG;
    float dcx = (G11 * hx - G01 * hy) * idG;
    float dcy = (G00 * hy - G01 * hx) * idG;
    float rhs = k0 + (hx * dcx + hy * dcy);
    if (!(rhs > 0.0f && rhs < 1e30f)) return 0;
    if (c->model == 0) {
        el[0] = c->fx * (v[0] * ivz + dcx) + c->cx;
        el[1] = c->fy * (v[1] * ivz + dcy) + c->cy;
        el[2] = G00 / (c->fx * c->fx);
        el[3] = G01 / (c->fx * c->fy);
        el[4] = G11 / (c->fy * c->fy);
        el[5] = rhs * 1.01f;
        el[6] = (-el[3]) / el[4];
        el[7] = (-el[3]) / el[2];
    } else {
        el[0] = dcx;
        el[1] = dcy;
        el[2] = G00;
        el[3] = G01;
        el[4] = G11;
        el[5] = sqrtf(rhs * 1.01f);
        el[6] = sqrtf(tG);
    }
    return 1;
}

/* Fisheye tile test: the tile's rays lie within gamma of its axis a, so their
 * gnomonic images lie within gamma / cos^2(phi + gamma) of a's (phi: the angle
 * of a from u), and with |x|_G <= sqrt(tr G) |x| a tile that reaches the
 * ellipse has |p_a - c|_G <= sqrt(threshold) + sqrt(tr G) gamma / cos^2(phi +
 * gamma), gamma <= 2 sin(gamma/2) / cos(gamma/2).  Evaluated multiplied through
 * by (a.u)^2, cos^4(phi + gamma) and cos^2(gamma/2), without division.  Tiles
 * reaching beyond cos(phi + gamma) = 0.2 are kept.  u: the rule record's
 * direction. */
static int fkb_test(const float *el, const float *u, const float *t) {
    float ca = (t[0] * u[0] + t[1] * u[1]) + t[2] * u[2];
    float s = t[3], ch = t[4];
    float sp = sqrtf(fmaxf(1.0f - ca * ca, 0.0f));
    float cg = 1.0f - 2.0f * (s * s);
    float sg = 2.0f * (s * ch);
    float cpg = ca * cg - sp * sg;
    if (!(cpg > 0.2f)) return 1;
    float e1x = el[7], e1y = el[8], e1z = el[9];
    float e2x = u[1] * e1z - u[2] * e1y;
    float e2y = u[2] * e1x - u[0] * e1z;
    float e2z = u[0] * e1y - u[1] * e1x;
    float nx = ((t[0] * e1x + t[1] * e1y) + t[2] * e1z) - el[0] * ca;
    float ny = ((t[0] * e2x + t[1] * e2y) + t[2] * e2z) - el[1] * ca;
    float Qn = nx * (el[2] * nx + 2.0f * (el[3] * ny)) + el[4] * (ny * ny);
    float c2 = cpg * cpg;
    float lhs = (Qn * (c2 * c2)) * (ch * ch);
    float r = (el[5] * c2) * ch + (2.0f * s) * el[6];
    return lhs <= (r * r) * (ca * ca);
}

/* Tile (tx, ty) against the ellipse: the minimum over the tile's pixel-centre
 * rectangle grown by `grow` pixels of (p - c)^T [[A,B],[B,C]] (p - c) is at most
 * q[0] (edges that separate the centre from the rectangle, clamped stationary
 * point along each). */
static int fell_test(const fcam *c, const float *e, const float *q, int tx, int ty, float grow) {
    float x0 = ((float)(TILE * tx) + 0.5f) - grow, y0 = ((float)(TILE * ty) + 0.5f) - grow;
    float x1 = fminf(((float)(TILE * tx) + (float)TILE) - 0.5f, (float)c->W - 0.5f) + grow;
    float y1 = fminf(((float)(TILE * ty) + (float)TILE) - 0.5f, (float)c->H - 0.5f) + grow;
    float dx0 = x0 - e[0], dx1 = x1 - e[0], dy0 = y0 - e[1], dy1 = y1 - e[1];
    int sx = dx0 > 0.0f || dx1 < 0.0f, sy = dy0 > 0.0f || dy1 < 0.0f;
    if (!sx && !sy) return 1;
    float best = 3.0e38f;
    if (sx) {
        float x = dx0 > 0.0f ? dx0 : dx1;
        float y = fminf(fmaxf(q[1] * x, dy0), dy1);
        best = x * (e[2] * x + 2.0f * (e[3] * y)) + e[4] * (y * y);
    }
    if (sy) {
        float y = dy0 > 0.0f ? dy0 : dy1;
        float x = fminf(fmaxf(q[2] * y, dx0), dx1);
        float b2 = x * (e[2] * x + 2.0f * (e[3] * y)) + e[4] * (y * y);
        best = fminf(best, b2);
    }
    return best <= q[0];
}

/* Per-Gaussian binning records [n*16] for one camera (FP32 inputs). */
void or_bin_gauss(const double *campk, int n, const float *means, const float *log_scales, const float *quats,
                  const float *logits, const float *rho2, float *recs) {
    fcam c;
    unpack_fcam(campk, &c);
#pragma omp parallel for schedule(static)
    for (int i = 0; i < n; ++i)
        fgauss(&c, means + 3 * (size_t)i, log_scales + 3 * (size_t)i, quats + 4 * (size_t)i, logits[i],
               rho2 ? rho2[i] : 0.0f, recs + 16 * (size_t)i);
}

/* Tile/Gaussian pair counts: per Gaussian (n) and per tile (ntiles); optional
 * dense pass matrix [n * ntiles] (bytes).  Returns the total pair count.  A
 * pair passes the cone test and, where it applies (pinhole cameras), the
 * silhouette ellipse built with the largest tile footprint bound m. */
long or_bin_counts(const double *campk, const float *table, int n, const float *recs, const float *means,
                   int *per_gauss, int *per_tile, unsigned char *pass) {
    fcam c;
    unpack_fcam(campk, &c);
    int ntx = (c.W + TILE - 1) / TILE;
    int nt = ntx * ((c.H + TILE - 1) / TILE);
    float mbar = 0.0f;
    for (int t = 0; t < nt; ++t) mbar = fmaxf(mbar, table[6 * (size_t)t + 5]);
    long total = 0;
    for (int t = 0; t < nt; ++t) per_tile[t] = 0;
    int *tcount = (int *)calloc((size_t)nt, sizeof(int));
#pragma omp parallel
    {
        int *mine = (int *)calloc((size_t)nt, sizeof(int));
#pragma omp for schedule(dynamic, 64) reduction(+ : total)
        for (int i = 0; i < n; ++i) {
            const float *g = recs + 16 * (size_t)i;
            float el[12];
            int ell = g[9] == 1.0f && fellipse(&c, g, means + 3 * (size_t)i, mbar, el);
            int cnt = 0;
            for (int t = 0; t < nt; ++t) {
                int ok = ftest(g, table + 6 * (size_t)t);
                if (ok && ell)
                    ok = c.model == 0 ? fell_test(&c, el, el + 5, t % ntx, t / ntx, 0.05f)
                                      : fkb_test(el, g, table + 6 * (size_t)t);
                if (pass) pass[(size_t)i * nt + t] = (unsigned char)ok;
                mine[t] += ok;
                cnt += ok;
            }
            per_gauss[i] = cnt;
            total += cnt;
        }
#pragma omp critical
        for (int t = 0; t < nt; ++t) tcount[t] += mine[t];
        free(mine);
    }
    for (int t = 0; t < nt; ++t) per_tile[t] = tcount[t];
    free(tcount);
    return total;
}

/* FP32 directions of a list of image points (the binning rule's ray function). */
void or_fdir(const double *campk, int npts, const float *xs, const float *ys, float *out, int *valid) {
    fcam c;
    unpack_fcam(campk, &c);
    for (int i = 0; i < npts; ++i) {
        valid[i] = fvalid(&c, xs[i], ys[i]);
        fdir(&c, xs[i], ys[i], out + 3 * (size_t)i);
    }
}

int or_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Threads of the following parallel loops (timing only: no result depends on it). */
void or_set_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}
