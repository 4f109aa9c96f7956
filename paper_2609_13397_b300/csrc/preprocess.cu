// K2: per-Gaussian preprocess.
//
// K2a (camera independent, run by set_scene): R from the normalised
// quaternion, s = exp(log s), the footprint floor of Eq. 10
// (s_eff = sqrt(s^2 + rho^2), sigma_eff = sigma prod s/s_eff) and the
// whitening W_eff = S_eff^-1 R^T of Sec. 3.
// K2b (per view, run by render): o_u = W_eff (o - mu), the SH colour seen
// along (mu - o)/|mu - o|, and the binning rule's direction / depth key.
// The raster record is 8 float4 per Gaussian:
//   [W row 0 | o_u.x] [W row 1 | o_u.y] [W row 2 | o_u.z] [rgb | sigma_eff]
//   [u | g0] [g1, g2, C00, C11] [C22, 2 C01, 2 C02, 2 C12] [rho^2, 0, 0, 0]
// (a flat Gaussian has [-rho^2, lo(o_u)] as its last word: see pair.cuh)
// where (u, g, C) define the pixel pre-test: with e = d - u, a pixel ray d
// with -1 + g.e + e^T C e > 0 cannot reach alpha >= 1/255 with this Gaussian.
// On pinhole views the words [4] and [5] hold that test's pixel-space ellipse
// instead, [c_x, c_y, G00, 2 G01] [G11, t, 0, 0] (pixel_cone_ellipse).
#include "pair.cuh"
#include "rule.cuh"
#include "sh.cuh"

namespace conegs {

__device__ __forceinline__ void quat_to_rot(float w, float x, float y, float z, float R[9]) {
    const float inv = rsqrtf(w * w + x * x + y * y + z * z);
    w *= inv; x *= inv; y *= inv; z *= inv;
    R[0] = 1.f - 2.f * (y * y + z * z); R[1] = 2.f * (x * y - w * z); R[2] = 2.f * (x * z + w * y);
    R[3] = 2.f * (x * y + w * z); R[4] = 1.f - 2.f * (x * x + z * z); R[5] = 2.f * (y * z - w * x);
    R[6] = 2.f * (x * z - w * y); R[7] = 2.f * (y * z + w * x); R[8] = 1.f - 2.f * (x * x + y * y);
}

__global__ void __launch_bounds__(256) scene_cache_kernel(SceneParams sp, float *__restrict__ Wout,
                                                          float *__restrict__ sig_eff) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= sp.n) return;
    float R[9];
    quat_to_rot(sp.quats[4 * i], sp.quats[4 * i + 1], sp.quats[4 * i + 2], sp.quats[4 * i + 3], R);
    const float rho2 = sp.rho2 ? sp.rho2[i] : 0.0f;
    const float logit = load_scalar(sp.logits, i, sp.storage);
    float sig = 1.0f / (1.0f + expf(-logit));
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const float s = expf(sp.log_scales[3 * i + a]);
        const float seff = sqrtf(s * s + rho2);
        sig *= s / seff;
        const float inv = 1.0f / seff;
#pragma unroll
        for (int b = 0; b < 3; ++b) Wout[9 * i + 3 * a + b] = R[3 * b + a] * inv;   // W_ab = R_ba / s_eff,a
    }
    sig_eff[i] = sig;
}


// Cone of pixel rays that can reach alpha >= 1/255 with a Gaussian.  Any such
// pair has q^T A^-1 q <= kappa^2 (det A >= 1, Eq. 9), which puts mu within
// kappa sqrt(s_max^2 + t*^2 m) of the pixel's centre ray (Sigma_render <=
// Sigma_fp,eff, Eq. 12; m >= (|delta_x|^2 + |delta_y|^2)/3), with t* bounded
// by min((L + kappa s_max)/(1 - kappa (1 + s_max/s_min) sqrt(m)), L + 255 kappa s_max).
// Returns sin and cos of half the cone's half-angle, inflated by `margin`
// (relative) + 1e-6; (1, 0) = every direction.
__device__ float2 cone_half_angle(float kap, float s2, float r1, float L, float m, float margin) {
    const float s = sqrtf(s2);
    const float c = kap * r1 * sqrtf(m);
    const float rfc = 255.0f * kap * s;
    float rf, tb;
    if (c < 1.0f) {
        const float tbf = (L + kap * s) / (1.0f - c);
        rf = fminf(kap * sqrtf(s2 + tbf * tbf * r1 * r1 * m), rfc);
        tb = fminf(tbf, L + rf);
    } else {
        rf = rfc;
        tb = L + rf;
    }
    if (L <= rf * (1.0f + margin)) return make_float2(1.0f, 0.0f);
    const float rp = kap * sqrtf(s2 + tb * tb * m);
    if (rp * (1.0f + margin) >= L) return make_float2(1.0f, 0.0f);
    const float sb = rp / L;
    const float sh2 = sb * sb / (2.0f * (1.0f + sqrtf(fmaxf(1.0f - sb * sb, 0.0f))));
    const float sbh = fminf(sqrtf(sh2) * (1.0f + margin) + 1e-6f, 1.0f);
    return make_float2(sbh, sqrtf(fmaxf(1.0f - sbh * sbh, 0.0f)));
}

// Visual-cone pre-test of the rasteriser.  A pair with alpha >= 1/255 has
// q^T A^-1 q <= kappa^2, kappa^2 = 2 ln(255 sigma) (det A >= 1, Eq. 9).  In
// world terms x = mu - x* (x* the closest-response point on the ray) lies in
// {x : x^T (Sigma_eff + F)^-1 x <= kappa^2} with F the world footprint
// (Eq. 12: Sigma_render <= Sigma_fp,eff), whose part across the ray is at most
// t*^2 m I (m at least the largest eigenvalue of [delta_i . delta_j]/3 over the
// view's pixels).  So the centre ray must meet the
// ellipsoid mu + {x : x^T M x <= 1}, M = (kappa'^2 (Sigma_eff + tau I))^-1,
// tau = t_b^2 m, kappa'^2 = 1.01 kappa^2 (margin for FP32 rounding).  The line
// o + t d meets it iff d^T C d <= 0, C = (1 - 1/v^T M v) M - (M v)(M v)^T / v^T M v,
// v = o - mu.  Expanded around u = -v/L (the direction of mu) with e = d - u:
//   L^2 d^T C d = -1 + 2 L e.(M v)/(v^T M v) + L^2 e^T C e,
// where the constant and linear terms are exact closed forms (u^T C u = -1/L^2,
// C u = M v/(L v^T M v)) and the quadratic term scales with |e|^2, so narrow
// cones of far, small Gaussians do not cancel in FP32.  With the rows w_i of
// W_eff (|w_i| = 1/s_i): M = sum_i c_i w_i w_i^T, c_i = 1/(kappa'^2 (1 + tau
// |w_i|^2)), w_i . v = (o_u)_i.  Output: g (3) and C' = L^2 C (6: 00 11 22,
// 2x 01 02 12).
__device__ void cone_quadric(const float W[9], const float ou[3], float kap2, float tau, float L, float g[3],
                             float C[6]) {
    float c[3], Mv[3] = {0.f, 0.f, 0.f}, vMv = 0.f;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        const float w2 = W[3 * i] * W[3 * i] + W[3 * i + 1] * W[3 * i + 1] + W[3 * i + 2] * W[3 * i + 2];
        c[i] = 1.0f / (kap2 * (1.0f + tau * w2));
        vMv += c[i] * ou[i] * ou[i];
#pragma unroll
        for (int k = 0; k < 3; ++k) Mv[k] += c[i] * ou[i] * W[3 * i + k];
    }
    if (!(vMv > 1.0f)) {            // optical centre inside the ellipsoid: every ray meets it
        g[0] = g[1] = g[2] = 0.0f;
        C[0] = C[1] = C[2] = C[3] = C[4] = C[5] = 0.0f;
        return;
    }
    const float a = 1.0f - 1.0f / vMv, b = 1.0f / vMv, L2 = L * L;
    float M[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};   // 00 11 22 01 02 12
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        const float *w = W + 3 * i;
        M[0] += c[i] * w[0] * w[0]; M[1] += c[i] * w[1] * w[1]; M[2] += c[i] * w[2] * w[2];
        M[3] += c[i] * w[0] * w[1]; M[4] += c[i] * w[0] * w[2]; M[5] += c[i] * w[1] * w[2];
    }
    C[0] = L2 * (a * M[0] - b * Mv[0] * Mv[0]);
    C[1] = L2 * (a * M[1] - b * Mv[1] * Mv[1]);
    C[2] = L2 * (a * M[2] - b * Mv[2] * Mv[2]);
    C[3] = 2.0f * L2 * (a * M[3] - b * Mv[0] * Mv[1]);
    C[4] = 2.0f * L2 * (a * M[4] - b * Mv[0] * Mv[2]);
    C[5] = 2.0f * L2 * (a * M[5] - b * Mv[1] * Mv[2]);
#pragma unroll
    for (int k = 0; k < 3; ++k) g[k] = 2.0f * L * b * Mv[k];
}

// Pinhole form of the same pre-test: the pixel centres whose rays meet the
// ellipsoid E = mu + {x : x^T M x <= 1} of cone_quadric (same M).  In the camera
// frame (m = R^T (mu - o), P = R^T M R, a = m^T P m, z = P m) the ray of direction
// d = m / m_z + delta, delta = (delta_x, delta_y, 0) on the plane z = 1, meets E iff
// (a - 1) d^T P d <= (d^T P m)^2, i.e.
//   delta^T G delta - 2 h^T delta <= k0,  G = (a - 1) P_xy - z_xy z_xy^T,
//   h = z_xy / m_z,  k0 = a / m_z^2
// (the constant and linear terms in delta cancel in closed form, so narrow cones
// of far, small Gaussians keep their digits); all three are scaled by 1/a here.
// With G positive definite this is the ellipse (delta - delta0)^T G (delta -
// delta0) <= k0 + h^T delta0, delta0 = G^-1 h; in pixels (delta = D (p - p_m),
// D = diag(1/f_x, 1/f_y), p_m the projection of mu) its centre is p_m + D^-1
// delta0 and its matrix D G D.  FP32 margins: the threshold x 1.01 (relative
// errors of the axes), then the ellipse grown by 0.02 px (rounding of the centre).
// Where the test does not apply (the camera within E, E reaching the camera
// plane, m_z <= 0) the record passes every pixel.  Output: r4 = (c_x, c_y, G00,
// 2 G01), r5 = (G11, t, 0, 0), the words pretest_pix reads.
__device__ void pixel_cone_ellipse(const CamParams &c, const float W[9], const float ou[3], float kap2, float tau,
                                   const float mu[3], float4 &r4, float4 &r5) {
    r4 = make_float4(0.f, 0.f, 0.f, 0.f);
    r5 = make_float4(0.f, 1.0f, 0.f, 0.f);            // pass every pixel
    const float v0 = mu[0] - c.o[0], v1 = mu[1] - c.o[1], v2 = mu[2] - c.o[2];
    const float mx = c.R[0] * v0 + c.R[3] * v1 + c.R[6] * v2;
    const float my = c.R[1] * v0 + c.R[4] * v1 + c.R[7] * v2;
    const float mz = c.R[2] * v0 + c.R[5] * v1 + c.R[8] * v2;
    if (!(mz > 0.0f)) return;
    float a = 0.f, P00 = 0.f, P01 = 0.f, P11 = 0.f, z0 = 0.f, z1 = 0.f;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        const float *w = W + 3 * i;
        const float w2 = w[0] * w[0] + w[1] * w[1] + w[2] * w[2];
        const float ci = 1.0f / (kap2 * (1.0f + tau * w2));
        const float wc0 = c.R[0] * w[0] + c.R[3] * w[1] + c.R[6] * w[2];   // R^T w_i, camera x and y
        const float wc1 = c.R[1] * w[0] + c.R[4] * w[1] + c.R[7] * w[2];
        a += ci * ou[i] * ou[i];                       // w_i . (mu - o) = -ou_i
        P00 += ci * wc0 * wc0;
        P01 += ci * wc0 * wc1;
        P11 += ci * wc1 * wc1;
        z0 -= ci * ou[i] * wc0;
        z1 -= ci * ou[i] * wc1;
    }
    if (!(a > 1.0f)) return;
    const float ia = 1.0f / a, b = 1.0f - ia;
    const float G00 = b * P00 - z0 * z0 * ia, G01 = b * P01 - z0 * z1 * ia, G11 = b * P11 - z1 * z1 * ia;
    const float det = G00 * G11 - G01 * G01;
    if (!(G00 > 0.0f && G11 > 0.0f && det > 0.0f)) return;
    const float imz = 1.0f / mz;
    const float h0 = z0 * ia * imz, h1 = z1 * ia * imz;
    const float idet = 1.0f / det;
    const float d0 = (G11 * h0 - G01 * h1) * idet, d1 = (G00 * h1 - G01 * h0) * idet;
    const float thr = imz * imz + h0 * d0 + h1 * d1;
    const float cxp = c.cx + c.fx * (mx * imz + d0), cyp = c.cy + c.fy * (my * imz + d1);
    const float ifx = 1.0f / c.fx, ify = 1.0f / c.fy;
    const float g00 = G00 * ifx * ifx, g01 = G01 * ifx * ify, g11 = G11 * ify * ify;
    const float grown = sqrtf(1.01f * fmaxf(thr, 0.0f)) + 0.02f * sqrtf(g00 + g11);
    const float t = grown * grown;
    if (!(isfinite(t) && isfinite(cxp) && isfinite(cyp) && isfinite(g00) && isfinite(g01) && isfinite(g11))) return;
    r4 = make_float4(cxp, cyp, g00, 2.0f * g01);
    r5 = make_float4(g11, t, 0.f, 0.f);
}

// t* bound of the binning rule (see cone_half_angle); false = no useful bound.
// rf: the bound on |x* - mu| (x* the ray's closest-response point) it came with.
__device__ bool tstar_bound(float kap, float s2, float r1, float L, float m, float &tb, float &rf) {
    const float s = sqrtf(s2);
    const float c = kap * r1 * sqrtf(m);
    const float rfc = 255.0f * kap * s;
    if (c < 1.0f) {
        const float tbf = (L + kap * s) / (1.0f - c);
        rf = fminf(kap * sqrtf(s2 + tbf * tbf * r1 * r1 * m), rfc);
        tb = fminf(tbf, L + rf);
    } else {
        rf = rfc;
        tb = L + rf;
    }
    tb *= 1.001f;
    return true;
}

// The footprint extremes (per unit depth) over the pixels a Gaussian can reach:
// the polar-angle bands of the view (see footprint_min_kernel) within beta of
// the angle of its direction u from the optical axis (beta: the half-angle of
// its binning cone, which holds every pixel ray it can reach alpha >= 1/255
// with), widened by 2e-3 rad for the rounding of both angles.  Empty bands
// are skipped; with none left, the view-wide values.
__device__ void footprint_range(const CamParams &c, const float *__restrict__ mcam, const float u[3], float2 gc,
                                float &mu_min, float &mu_max) {
    const float *bmin = mcam + FP_MIN + 1, *bmax = mcam + FP_MAX + 1;
    int j0 = 0, j1 = FP_BANDS - 1;
    if (gc.x < 1.0f) {
        const float cz = u[0] * c.R[2] + u[1] * c.R[5] + u[2] * c.R[8];
        const float th = acosf(fminf(fmaxf(cz, -1.0f), 1.0f));
        const float beta = 2.0f * asinf(gc.x) + 2e-3f;
        const float band_scale = (float)FP_BANDS / 3.14159265f;
        j0 = max(0, (int)floorf((th - beta) * band_scale));
        j1 = min(FP_BANDS - 1, (int)floorf((th + beta) * band_scale));
    }
    unsigned int lo = 0xffffffffu, hi = 0u;
    for (int j = j0; j <= j1; ++j) {
        const unsigned int a = __float_as_uint(bmin[j]), b = __float_as_uint(bmax[j]);
        lo = min(lo, a);        // non-negative floats order as their bits; empty: 0xffffffff
        hi = max(hi, b);        // empty: 0
    }
    const unsigned int glo = __float_as_uint(mcam[FP_MIN]);
    mu_min = __uint_as_float(lo != 0xffffffffu ? lo : (glo != 0xffffffffu ? glo : 0u));
    mu_max = hi != 0u ? __uint_as_float(hi) : mcam[FP_MAX];
}

// Per view: binning direction/depth (the FP32 rule) and the raster record.
// Latency-bound (one Gaussian per thread, dependent loads and transcendental
// chains): four CTAs per SM (64 registers, a few bytes of spill) run it faster
// than three at the 79 registers it would otherwise take.
__global__ void __launch_bounds__(256, 4) view_records_kernel(CamParams c, SceneParams sp, const float *__restrict__ mcam,
                                                           float mzf, int fov_cull, int pretest, int pixtest,
                                                           int dilute,
                                                           float4 *__restrict__ rec, float4 *__restrict__ gview,
                                                           float2 *__restrict__ gcone,
                                                           uint8_t *__restrict__ gflag,
                                                           float4 *__restrict__ gell,
                                                           unsigned long long *__restrict__ nflat,
                                                           uint8_t *__restrict__ gflat) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= sp.n) return;
    gflat[i] = 0;
    const float mu[3] = {sp.means[3 * i], sp.means[3 * i + 1], sp.means[3 * i + 2]};
    float flag = sp.binrec[BINREC * i + 5], u[3], L;
    rule_gauss_view(c, mu, flag, u, L);
    gview[i] = make_float4(u[0], u[1], u[2], L);
    const float m = fmaxf(*mcam, mzf);   // footprint bound (raised for the z/f variant)
    // binning prefilter: the cone of the binning rule's own bound (its kappa and
    // scale bounds), camera-wide footprint, wide margin
    const float *br = sp.binrec + BINREC * i;
    const float2 gc = flag != 0.0f && L > 0.0f ? cone_half_angle(br[0], br[4], sqrtf(br[3]), L, m, 1e-3f)
                                               : make_float2(1.0f, 0.0f);
    gcone[i] = gc;
    if (fov_cull && flag == 1.0f && gc.y > 1e-3f) {
        // outside the camera's cone: every tile cone lies within mcam[19] of the
        // optical axis, the Gaussian's within beta of u, so no tile can keep it
        const float cz = u[0] * c.R[2] + u[1] * c.R[5] + u[2] * c.R[8];
        const float ang = acosf(fminf(fmaxf(cz, -1.0f), 1.0f));
        if (ang > 2.0f * asinf(fminf(gc.x, 1.0f)) + mcam[19] + 2e-3f) flag = 0.0f;
    }
    gflag[i] = (uint8_t)flag;
    if (flag == 0.0f) return;
    float W[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) W[k] = sp.W[9 * i + k];
    const float w0 = c.o[0] - mu[0], w1 = c.o[1] - mu[1], w2 = c.o[2] - mu[2];
    float ou[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) ou[a] = W[3 * a] * w0 + W[3 * a + 1] * w1 + W[3 * a + 2] * w2;
    // SH colour along (mu - o)/|mu - o|
    float dx = u[0], dy = u[1], dz = u[2];
    if (!(L > 0.0f)) { dx = 0.f; dy = 0.f; dz = 1.f; }
    float Y[16];
    sh_basis(dx, dy, dz, sp.sh_degree, Y);
    float col[3];
    sh_colour(sp.sh, i, sp.sh_degree, sp.storage, Y, col);
    const float rho2 = sp.rho2 ? sp.rho2[i] : 0.0f;
    // the binning rule's silhouette ellipse (threshold -1 when it does not apply)
    {
        float el[ELL_F] = {0.f, 0.f, 0.f, 0.f, 0.f, -1.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        if (!(flag == 1.0f && rule_ellipse(c, br, L, mu, br + 6, m, el))) el[5] = -1.0f;
        float4 *ge = gell + 3 * i;
        ge[0] = make_float4(el[0], el[1], el[2], el[3]);
        ge[1] = make_float4(el[4], el[5], el[6], el[7]);
        ge[2] = make_float4(el[8], el[9], el[10], el[11]);
    }
    // rasteriser pre-test, with the exact kappa^2 = 2 ln(255 sigma): its ray-direction
    // form (u, g, C), or on pinhole views (pixtest) the pixel-space ellipse.
    // The ellipsoid is that of Sigma_eff + tau I, tau = t_b^2 mu_max (mu_max: the
    // largest per-unit-depth footprint eigenvalue over the pixels the Gaussian
    // can reach, footprint_range; t_b >= t*): the
    // whitened footprint M_perp W (t*^2 sum_i delta_i delta_i^T / 3) W^T M_perp is
    // at most tau M_perp W W^T M_perp, so q^T A^-1 q is at least the ray's
    // distance in the metric of I + tau W W^T.
    // With `dilute`, the footprint's dilution of the peak narrows it.  Clamped by
    // the floor (Eq. 12), the world footprint Sigma_render has eigenvalues
    // (lambda_j - rho^2)_+, with both lambda_j >= t*^2 mu_min (the smallest
    // per-unit-depth footprint over the same pixels); the two non-zero eigenvalues nu_k of W
    // Sigma_render W^T then have nu_1 + nu_2 >= c (1/s_max^2 + 1/s_mid^2) and
    // nu_1 nu_2 >= c^2 / (s_max^2 s_mid^2) (interlacing of the compression of W^T W,
    // whose eigenvalues are 1/s_eff,a^2), c = (t*^2 mu_min - rho^2)_+, so that
    // det A >= (1 + c/s_max^2)(1 + c/s_mid^2).  With t* >= L - r_f (r_f bounding
    // |x* - mu|), a pair reaching alpha >= 1/255 has
    // q^T A^-1 q <= 2 ln(255 sigma_eff) - ln(1 + c/s_max^2) - ln(1 + c/s_mid^2).
    float g[3] = {0.f, 0.f, 0.f}, C[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    float pu[3] = {dx, dy, dz};
    float4 pix4 = make_float4(0.f, 0.f, 0.f, 0.f), pix5 = make_float4(0.f, -1.0f, 0.f, 0.f);   // rejects every pixel
    if (!pretest) {
        pix5 = make_float4(0.f, 1.0f, 0.f, 0.f);        // every pixel (g = C = 0: every ray)
    } else {
        const float sig = 1.0f / (1.0f + expf(-load_scalar(sp.logits, i, sp.storage)));
        const float k2 = 2.0f * logf(255.0f * sig);
        const float l0 = sp.log_scales[3 * i], l1 = sp.log_scales[3 * i + 1], l2 = sp.log_scales[3 * i + 2];
        const float lmax = fmaxf(fmaxf(l0, l1), l2), lmin = fminf(fminf(l0, l1), l2);
        const float lmid = fmaxf(fminf(l0, l1), fminf(fmaxf(l0, l1), l2));
        const float s2 = expf(2.0f * lmax) * 1.00001f + rho2, s2mn = expf(2.0f * lmin) * 0.99999f + rho2;
        // footprint extremes per unit depth over the pixels the Gaussian can reach;
        // the ellipsoid's bound is the largest eigenvalue, or the z/f variant's own
        float mu_lo, mu_hi;
        footprint_range(c, mcam, u, gc, mu_lo, mu_hi);
        const float mlam = fmaxf(mu_hi * 1.01f, mzf);
        if (!(k2 > 0.0f)) {
            // sigma < 1/255: never reaches the alpha cut (value 99 for every unit d)
            pu[0] = pu[1] = pu[2] = 0.0f;
            C[0] = C[1] = C[2] = 100.0f;
        } else if (L > 0.0f) {
            float tb, rf;
            // s_max / s_min: the world half-edges are f = (I - d w^T) delta with
            // |I - d w^T| <= (r + 1/r)/2 (Kantorovich), so the world footprint's
            // largest eigenvalue is at most ((r + 1/r)/2)^2 t*^2 mlam: the t* bound
            // holds with mlam in place of the rule's trace bound m
            const float rr = sqrtf(s2 / s2mn);
            tstar_bound(sqrtf(k2), s2, fmaxf(0.5f * (rr + 1.0f / rr) * 1.00001f, 1.0f), L, mlam, tb, rf);
            float kq2 = k2;
            if (dilute) {
                const float mumin = fmaxf(mu_lo, 0.0f) * 0.99f;
                const float tlo = fmaxf(L - rf * 1.001f, 0.0f);
                const float cf = fmaxf(tlo * tlo * mumin - rho2 * 1.001f, 0.0f);
                const float s2md = expf(2.0f * lmid) * 1.00001f + rho2;
                kq2 = 2.0f * logf(255.0f * sp.sig_eff[i] * 1.0001f) -
                      0.999f * (log1pf(cf / s2) + log1pf(cf / s2md));
            }
            if (!(kq2 > 0.0f)) {
                // the footprint dilutes this Gaussian below the alpha cut in this view
                pu[0] = pu[1] = pu[2] = 0.0f;
                C[0] = C[1] = C[2] = 100.0f;
            } else if (pixtest) {
                pixel_cone_ellipse(c, W, ou, 1.01f * kq2, tb * tb * mlam * 1.001f, mu, pix4, pix5);
            } else {
                cone_quadric(W, ou, 1.01f * kq2, tb * tb * mlam * 1.001f, L, g, C);
            }
        } else {
            pix5 = make_float4(0.f, 1.0f, 0.f, 0.f);     // mu at the optical centre: every pixel
        }
    }
    // flat Gaussian (s_eff,max / s_eff,min > FLAT_RATIO): the response is taken in
    // FP64 from o_u = hi + lo, formed here in FP64 from the FP32 W, o and mu; the
    // record marks it by the sign bit of its rho^2 word
    float4 r7 = make_float4(rho2, 0.f, 0.f, 0.f);
    {
        const float lmax = fmaxf(fmaxf(sp.log_scales[3 * i], sp.log_scales[3 * i + 1]), sp.log_scales[3 * i + 2]);
        const float lmin = fminf(fminf(sp.log_scales[3 * i], sp.log_scales[3 * i + 1]), sp.log_scales[3 * i + 2]);
        const float s2max = expf(2.0f * lmax) + rho2, s2min = expf(2.0f * lmin) + rho2;
        if (s2max > FLAT_RATIO * FLAT_RATIO * s2min) {
            const double v0 = (double)c.o[0] - (double)mu[0], v1 = (double)c.o[1] - (double)mu[1],
                         v2 = (double)c.o[2] - (double)mu[2];
            float lo[3];
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                const double o64 = (double)W[3 * a] * v0 + (double)W[3 * a + 1] * v1 + (double)W[3 * a + 2] * v2;
                ou[a] = (float)o64;
                lo[a] = (float)(o64 - (double)ou[a]);
            }
            r7 = make_float4(-rho2, lo[0], lo[1], lo[2]);
            gflat[i] = 1;
            atomicAdd(nflat, 1ull);
        }
    }
    float4 *r = rec + (size_t)REC_F4 * i;
    r[0] = make_float4(W[0], W[1], W[2], ou[0]);
    r[1] = make_float4(W[3], W[4], W[5], ou[1]);
    r[2] = make_float4(W[6], W[7], W[8], ou[2]);
    r[3] = make_float4(col[0], col[1], col[2], sp.sig_eff[i]);
    if (pixtest) {
        r[4] = pix4;
        r[5] = pix5;
        r[6] = make_float4(0.f, 0.f, 0.f, 0.f);
    } else {
        r[4] = make_float4(pu[0], pu[1], pu[2], g[0]);
        r[5] = make_float4(g[1], g[2], C[0], C[1]);
        r[6] = make_float4(C[2], C[3], C[4], C[5]);
    }
    r[7] = r7;
}

cudaError_t launch_scene_cache(const SceneParams &sp, float *W, float *sig_eff, cudaStream_t s) {
    if (sp.n == 0) return cudaSuccess;
    scene_cache_kernel<<<(unsigned)div_up(sp.n, 256), 256, 0, s>>>(sp, W, sig_eff);
    note_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_view_records(const CamParams &c, const SceneParams &sp, const float *mcam, float mzf,
                                int fov_cull, int pretest, int pixtest, int dilute, float4 *rec, float4 *gview,
                                float2 *gcone,
                                uint8_t *gflag,
                                float4 *gell, unsigned long long *nflat, uint8_t *gflat, cudaStream_t s) {
    if (sp.n == 0) return cudaSuccess;
    view_records_kernel<<<(unsigned)div_up(sp.n, 256), 256, 0, s>>>(c, sp, mcam, mzf, fov_cull, pretest, pixtest,
                                                                    dilute, rec,
                                                                    gview, gcone, gflag, gell, nflat, gflat);
    note_launches(1);
    return cudaGetLastError();
}

}  // namespace conegs
