// FP32 binning-rule primitives (see binning.cu for the rule).  Every
// operation is one correctly rounded FP32 operation through an explicit _rn
// intrinsic, evaluated in the order written, so the rule's decisions are the
// same bits on every build and in any reference that follows the same
// operation sequence.
#pragma once
#include "common.cuh"

namespace conegs {

__device__ __forceinline__ float r_add(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float r_sub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float r_mul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float r_div(float a, float b) { return __fdiv_rn(a, b); }
__device__ __forceinline__ float r_sqrt(float a) { return __fsqrt_rn(a); }

// ---------------------------------------------------------------- FP32 rule primitives

__device__ __forceinline__ bool rule_valid(const CamParams &c, float x, float y) {
    if (c.model == 0) return true;
    float a = r_div(r_sub(x, c.cx), c.fx);
    float b = r_div(r_sub(y, c.cy), c.fy);
    float r2 = r_add(r_mul(a, a), r_mul(b, b));
    return r2 <= c.rlim2;
}

__device__ __forceinline__ void rule_sincos(float t, float &sn, float &cs) {
    const float S1 = (float)(-1.0 / 6.0), S2 = (float)(1.0 / 120.0), S3 = (float)(-1.0 / 5040.0),
                S4 = (float)(1.0 / 362880.0), S5 = (float)(-1.0 / 39916800.0),
                S6 = (float)(1.0 / 6227020800.0), S7 = (float)(-1.0 / 1307674368000.0),
                S8 = (float)(1.0 / 355687428096000.0);
    const float C1 = (float)(-1.0 / 2.0), C2 = (float)(1.0 / 24.0), C3 = (float)(-1.0 / 720.0),
                C4 = (float)(1.0 / 40320.0), C5 = (float)(-1.0 / 3628800.0), C6 = (float)(1.0 / 479001600.0),
                C7 = (float)(-1.0 / 87178291200.0), C8 = (float)(1.0 / 20922789888000.0);
    float t2 = r_mul(t, t);
    float s = S8;
    s = r_add(r_mul(s, t2), S7); s = r_add(r_mul(s, t2), S6); s = r_add(r_mul(s, t2), S5); s = r_add(r_mul(s, t2), S4);
    s = r_add(r_mul(s, t2), S3); s = r_add(r_mul(s, t2), S2); s = r_add(r_mul(s, t2), S1); s = r_add(r_mul(s, t2), 1.0f);
    sn = r_mul(s, t);
    float c = C8;
    c = r_add(r_mul(c, t2), C7); c = r_add(r_mul(c, t2), C6); c = r_add(r_mul(c, t2), C5); c = r_add(r_mul(c, t2), C4);
    c = r_add(r_mul(c, t2), C3); c = r_add(r_mul(c, t2), C2); c = r_add(r_mul(c, t2), C1); c = r_add(r_mul(c, t2), 1.0f);
    cs = c;
}

static __device__ __noinline__ void rule_dir(const CamParams &c, float x, float y, float out[3]) {
    float a = r_div(r_sub(x, c.cx), c.fx);
    float b = r_div(r_sub(y, c.cy), c.fy);
    float v0, v1, v2;
    if (c.model == 0) {
        float n2 = r_add(r_add(r_mul(a, a), r_mul(b, b)), 1.0f);
        float s = r_sqrt(n2);
        v0 = r_div(a, s); v1 = r_div(b, s); v2 = r_div(1.0f, s);
    } else {
        float r2 = r_add(r_mul(a, a), r_mul(b, b));
        float r = r_sqrt(r2);
        float th = fminf(r, c.thlim);
        for (int it = 0; it < 12; ++it) {
            float t2 = r_mul(th, th);
            float p = r_add(r_mul(r_add(r_mul(r_add(r_mul(c.k[3], t2), c.k[2]), t2), c.k[1]), t2), c.k[0]);
            float f = r_sub(r_mul(th, r_add(1.0f, r_mul(t2, p))), r);
            float dp = r_add(r_mul(r_add(r_mul(r_add(r_mul(r_mul(9.0f, c.k[3]), t2), r_mul(7.0f, c.k[2])), t2), r_mul(5.0f, c.k[1])), t2),
                          r_mul(3.0f, c.k[0]));
            float fp = r_add(1.0f, r_mul(t2, dp));
            th = r_sub(th, r_div(f, fp));
            th = fminf(fmaxf(th, 0.0f), c.thlim);
        }
        float sn, cs;
        rule_sincos(th, sn, cs);
        if (r > 0.0f) {
            v0 = r_div(r_mul(sn, a), r);
            v1 = r_div(r_mul(sn, b), r);
        } else {
            v0 = 0.0f;
            v1 = 0.0f;
        }
        v2 = cs;
    }
#pragma unroll
    for (int i = 0; i < 3; ++i) out[i] = r_add(r_add(r_mul(c.R[3 * i], v0), r_mul(c.R[3 * i + 1], v1)), r_mul(c.R[3 * i + 2], v2));
}

static __device__ void rule_edge(const CamParams &c, float x, float y, const float d[3], int axis, float e[3]) {
    float xp = axis == 0 ? r_add(x, 0.5f) : x, yp = axis == 1 ? r_add(y, 0.5f) : y, t[3];
    if (rule_valid(c, xp, yp)) {
        rule_dir(c, xp, yp, t);
#pragma unroll
        for (int i = 0; i < 3; ++i) e[i] = r_sub(t[i], d[i]);
    } else {
        float xm = axis == 0 ? r_sub(x, 0.5f) : x, ym = axis == 1 ? r_sub(y, 0.5f) : y;
        rule_dir(c, xm, ym, t);
#pragma unroll
        for (int i = 0; i < 3; ++i) e[i] = r_sub(d[i], t[i]);
    }
}

// exp(x) = 2^k sum_{j<=9} f^j/j!, x = k ln2 + f (relative error < 1e-5 on [-80, 80]).
__device__ __forceinline__ float rule_exp(float x) {
    const float INV_LN2 = (float)(1.0 / 0.69314718055994530942), LN2F = (float)0.69314718055994530942;
    const float E2 = (float)(1.0 / 2.0), E3 = (float)(1.0 / 6.0), E4 = (float)(1.0 / 24.0),
                E5 = (float)(1.0 / 120.0), E6 = (float)(1.0 / 720.0), E7 = (float)(1.0 / 5040.0),
                E8 = (float)(1.0 / 40320.0), E9 = (float)(1.0 / 362880.0);
    x = fminf(fmaxf(x, -80.0f), 80.0f);
    float kf = floorf(r_mul(x, INV_LN2));
    float f = r_sub(x, r_mul(kf, LN2F));
    float p = E9;
    p = r_add(r_mul(p, f), E8); p = r_add(r_mul(p, f), E7); p = r_add(r_mul(p, f), E6); p = r_add(r_mul(p, f), E5);
    p = r_add(r_mul(p, f), E4); p = r_add(r_mul(p, f), E3); p = r_add(r_mul(p, f), E2); p = r_add(r_mul(p, f), 1.0f);
    p = r_add(r_mul(p, f), 1.0f);
    int k = (int)kf;
    float two = __uint_as_float((uint32_t)(k + 127) << 23);
    return r_mul(p, two);
}

// Scene-level part of the Gaussian bound: kap, ks, kr, r1sq, s2, flag
// (flag 0: sigma < 1/255, never contributes; 1: normal).
static __device__ void rule_gauss_scene(const float ls[3], float logit, float rho2, float rec[6]) {
    const float K255 = 11.082528f;   // >= 2 ln 255
    const float LN2LO = 0.6931471f;  // <= ln 2
    float lmax = fmaxf(fmaxf(ls[0], ls[1]), ls[2]);
    float lmin = fminf(fminf(ls[0], ls[1]), ls[2]);
    float s2 = r_add(r_mul(rule_exp(r_mul(2.0f, lmax)), 1.0001f), rho2);
    float s2mn = r_add(r_mul(rule_exp(r_mul(2.0f, lmin)), 0.9999f), rho2);
    float kap2 = r_sub(K255, r_mul(2.0f, fmaxf(fmaxf(0.0f, -logit), r_sub(LN2LO, r_mul(0.5f, logit)))));
    if (!(kap2 > 0.0f)) {
        rec[0] = rec[1] = rec[2] = rec[3] = rec[4] = 0.0f;
        rec[5] = 0.0f;
        return;
    }
    float kap = r_sqrt(kap2);
    float s = r_sqrt(s2);
    // r1 bounds |f_i| / |delta_i| for the world half-edges f_i = delta_i - c_i d of
    // Eq. 6 mapped back by W^-1: their part across d is delta_i's own, their part
    // along d at most beta |delta_i| with beta = max |P_perp S^-1 d| / (d^T S^-1 d)
    // = (r - 1/r) / 2, r = s_max / s_min (S = Sigma_eff), so r1 = sqrt(1 + beta^2)
    // = (r + 1/r) / 2 (with a relative margin for the rounding)
    float rr = r_div(s, r_sqrt(s2mn));
    float r1 = fmaxf(r_mul(r_mul(r_add(rr, r_div(1.0f, rr)), 0.5f), 1.00001f), 1.0f);
    rec[0] = kap;
    rec[1] = r_mul(kap, s);
    rec[2] = r_mul(kap, r1);
    rec[3] = r_mul(r1, r1);
    rec[4] = s2;
    rec[5] = 1.0f;
}

// View-level part: unit direction u = (mu - o)/L and L; flag 2 = pass-all.
__device__ __forceinline__ void rule_gauss_view(const CamParams &c, const float mu[3], float &flag, float u[3],
                                                float &L) {
    float v0 = r_sub(mu[0], c.o[0]), v1 = r_sub(mu[1], c.o[1]), v2 = r_sub(mu[2], c.o[2]);
    float L2 = r_add(r_add(r_mul(v0, v0), r_mul(v1, v1)), r_mul(v2, v2));
    L = r_sqrt(L2);
    u[0] = u[1] = u[2] = 0.0f;
    if (flag == 0.0f) return;
    if (!(L > 0.0f)) {
        flag = 2.0f;
        return;
    }
    u[0] = r_div(v0, L); u[1] = r_div(v1, L); u[2] = r_div(v2, L);
}

// The Gaussian's side of the rule at footprint bound m: sin and cos of half
// the half-angle beta of its cone (sbh, cbh).  Returns true when every valid
// tile passes at this m (L <= r_f or r_p >= L).  The rule is monotone in m.
__device__ __forceinline__ bool rule_half(const float *g, const float L, const float m, float &sbh, float &cbh) {
    const float kap = g[0], ks = g[1], kr = g[2], r1sq = g[3], s2 = g[4];
    float sm = r_sqrt(m);
    float cc = r_mul(kr, sm);
    // two valid bounds on |x* - mu| and t*, combined by min (monotone in m)
    float rfc = r_mul(255.0f, ks);
    float tb, rf;
    if (cc < 1.0f) {
        float tbf = r_div(r_add(L, ks), r_sub(1.0f, cc));
        float rff = r_mul(kap, r_sqrt(r_add(s2, r_mul(r_mul(r_mul(tbf, tbf), r1sq), m))));
        rf = fminf(rff, rfc);
        tb = fminf(tbf, r_add(L, rf));
    } else {
        rf = rfc;
        tb = r_add(L, rf);
    }
    if (L <= rf) return true;
    float rp = r_mul(kap, r_sqrt(r_add(s2, r_mul(r_mul(tb, tb), m))));
    if (rp >= L) return true;
    float sb = r_div(rp, L);
    float cb = r_sqrt(r_sub(1.0f, r_mul(sb, sb)));
    float sh2 = r_div(r_mul(sb, sb), r_mul(2.0f, r_add(1.0f, cb)));
    sbh = r_sqrt(sh2);
    cbh = r_sqrt(r_sub(1.0f, sh2));
    return false;
}

// The per (Gaussian, tile) test.  g: scene rec (kap ks kr r1sq s2 flag); gv: u0 u1 u2 L.
__device__ __forceinline__ bool rule_test(const float *g, const float4 gv, const float *t) {
    if (t[3] < 0.0f) return false;
    if (g[5] == 0.0f) return false;
    if (g[5] == 2.0f) return true;
    float sbh, cbh;
    if (rule_half(g, gv.w, t[5], sbh, cbh)) return true;
    float sphi = r_add(r_mul(sbh, t[4]), r_mul(cbh, t[3]));
    float e0 = r_sub(gv.x, t[0]), e1 = r_sub(gv.y, t[1]), e2 = r_sub(gv.z, t[2]);
    float ch2 = r_add(r_add(r_mul(e0, e0), r_mul(e1, e1)), r_mul(e2, e2));
    float lim = r_add(r_mul(r_mul(2.0f, sphi), 1.0001f), 4e-6f);
    return ch2 <= r_mul(lim, lim);
}


// The same test evaluated with fast arithmetic (FMA contraction, SFU
// reciprocal square roots and divisions).  Returns 1 (the exact rule passes),
// 0 (the exact rule fails) or 2 (too close to a branch or to the final
// comparison to tell: evaluate rule_test).  The bands are far wider than the
// fast chain's rounding error (~1e-5 relative once the cancellations at
// c -> 1 and sin(beta) -> 1 are excluded), so a 0/1 answer is always the
// exact rule's.
__device__ __forceinline__ int rule_test_fast(const float *g, const float4 gv, const float *t) {
    if (t[3] < 0.0f) return 0;
    if (g[5] == 0.0f) return 0;
    if (g[5] == 2.0f) return 1;
    const float L = gv.w, kap = g[0], ks = g[1], kr = g[2], r1sq = g[3], s2 = g[4];
    const float m = t[5];
    const float sm = m > 0.0f ? m * rsqrtf(m) : 0.0f;
    const float cc = kr * sm;
    if (fabsf(cc - 1.0f) < 1e-2f) return 2;
    const float rfc = 255.0f * ks;
    float tb, rf;
    if (cc < 1.0f) {
        const float tbf = __fdividef(L + ks, 1.0f - cc);
        const float x = s2 + tbf * tbf * r1sq * m;
        const float rff = kap * x * rsqrtf(x);
        rf = fminf(rff, rfc);
        tb = fminf(tbf, L + rf);
    } else {
        rf = rfc;
        tb = L + rf;
    }
    if (L < rf * (1.0f - 1e-3f)) return 1;
    if (L <= rf * (1.0f + 1e-3f)) return 2;
    const float y = s2 + tb * tb * m;
    const float rp = kap * y * rsqrtf(y);
    if (rp > L * (1.0f + 1e-3f)) return 1;
    if (rp >= L * (1.0f - 1e-2f)) return 2;
    const float sb = __fdividef(rp, L);
    const float om = 1.0f - sb * sb;
    const float cb = om * rsqrtf(om);
    const float sh2 = __fdividef(sb * sb, 2.0f * (1.0f + cb));
    const float sbh = sh2 * rsqrtf(sh2);
    const float oh = 1.0f - sh2;
    const float cbh = oh * rsqrtf(oh);
    const float sphi = sbh * t[4] + cbh * t[3];
    const float e0 = gv.x - t[0], e1 = gv.y - t[1], e2 = gv.z - t[2];
    const float ch2 = e0 * e0 + e1 * e1 + e2 * e2;
    const float lim = 2.0f * sphi * 1.0001f + 4e-6f;
    const float l2 = lim * lim;
    if (ch2 < l2 * (1.0f - 1e-4f) - 1e-12f) return 1;
    if (ch2 > l2 * (1.0f + 1e-4f) + 1e-12f) return 0;
    return 2;
}

// A tile the exact rule certainly keeps: its axis lies inside the Gaussian's
// cone at a footprint bound m_lo no larger than the tile's own (sbh_lo, cbh_lo
// from rule_half at m_lo; sbh_lo = RULE_ALL when every valid tile passes at
// m_lo), with a relative margin of 1e-5.  The rule is monotone in m, and
// sin((beta + gamma)/2) grows with beta while (beta + gamma)/2 stays below 90
// degrees (beta <= 90, tile cones below 90 degrees here); the margin is far
// above the rounding of this test and of the rule's chain (both
// well-conditioned here: sphi is a sum of non-negative terms).
// sbh_lo = RULE_NONE: no such bound (the test never decides).
constexpr float RULE_ALL = 1e30f, RULE_NONE = -1.0f;
__device__ __forceinline__ bool rule_pass_lo(const float sbh_lo, const float cbh_lo, const float4 gv, const float *t) {
    if (t[3] < 0.0f || sbh_lo < 0.0f) return false;
    if (sbh_lo == RULE_ALL) return true;
    if (t[3] > 0.7f) return false;
    const float e0 = gv.x - t[0], e1 = gv.y - t[1], e2 = gv.z - t[2];
    const float ch2 = e0 * e0 + e1 * e1 + e2 * e2;
    const float lim = (2.0f * 1.0001f) * (sbh_lo * t[4] + cbh_lo * t[3]) + 4e-6f;
    return ch2 <= lim * lim * 0.99999f;
}

// (sbh_lo, cbh_lo) of rule_pass_lo for a Gaussian with scene record g (flag
// g[5]) at the view's smallest footprint bound m_lo.
__device__ __forceinline__ float2 rule_lo(const float *g, const float L, const float m_lo) {
    if (g[5] == 2.0f) return make_float2(RULE_ALL, 0.0f);
    if (g[5] != 1.0f || !(m_lo >= 0.0f && m_lo < 1e30f)) return make_float2(RULE_NONE, 0.0f);
    float sbh, cbh;
    if (rule_half(g, L, m_lo, sbh, cbh)) return make_float2(RULE_ALL, 0.0f);
    return make_float2(sbh, cbh);
}

// ---------------------------------------------------------------- silhouette ellipse (pinhole cameras)
//
// A contributing pair's ray passes through the ellipsoid
//   E = {x : (x - mu)^T C^-1 (x - mu) <= kap^2},  C = Sigma_eff + t_b^2 m I
// (Eq. 9 and 12: A >= I, the rendered footprint is at most t*^2 m I, t* <= t_b),
// and the lines through the camera centre that meet E form an elliptic cone
// whose trace on a pinhole's image plane is an ellipse.  With the scene
// scaled by 1/L about the camera centre (v = (mu - o)/L, L = |mu - o|) and C
// normalised by its mean eigenvalue tau, a line of direction d = (x, y, 1)
// meets E iff, for delta = d - v/v_z,
//   delta^T G delta - 2 h^T delta <= k0,  G = (a - k^2) Ci_xy - w_xy w_xy^T,
//   h = k^2 w_xy / v_z,  k0 = k^2 a / v_z^2,  w = Ci v,  a = v^T w,  k^2 = kap^2 tau / L^2.
// The rule keeps a tile only when this ellipse (rhs widened by 1%, the tile's
// pixel-centre rectangle by 0.05 px, C by 1e-4 tau I) meets the rectangle.  It
// applies when the camera lies outside E with margin, E is seen within ~77
// degrees of the axis and the ellipse's aspect is below 1000; otherwise the
// cone test alone decides.

constexpr int ELL_F = 12;          // floats per Gaussian of the silhouette record

// Scene part: Sigma_eff = R diag(s_eff^2) R^T (xx xy xz yy yz zz),
// s_eff^2 = exp(2 log s) * 1.0001 + rho^2.
static __device__ void rule_gauss_sigma(const float q[4], const float ls[3], float rho2, float S[6]) {
    const float n2 = r_add(r_add(r_add(r_mul(q[0], q[0]), r_mul(q[1], q[1])), r_mul(q[2], q[2])), r_mul(q[3], q[3]));
    const float inv = r_div(1.0f, r_sqrt(n2));
    const float w = r_mul(q[0], inv), x = r_mul(q[1], inv), y = r_mul(q[2], inv), z = r_mul(q[3], inv);
    float R[9];
    R[0] = r_sub(1.0f, r_mul(2.0f, r_add(r_mul(y, y), r_mul(z, z))));
    R[1] = r_mul(2.0f, r_sub(r_mul(x, y), r_mul(w, z)));
    R[2] = r_mul(2.0f, r_add(r_mul(x, z), r_mul(w, y)));
    R[3] = r_mul(2.0f, r_add(r_mul(x, y), r_mul(w, z)));
    R[4] = r_sub(1.0f, r_mul(2.0f, r_add(r_mul(x, x), r_mul(z, z))));
    R[5] = r_mul(2.0f, r_sub(r_mul(y, z), r_mul(w, x)));
    R[6] = r_mul(2.0f, r_sub(r_mul(x, z), r_mul(w, y)));
    R[7] = r_mul(2.0f, r_add(r_mul(y, z), r_mul(w, x)));
    R[8] = r_sub(1.0f, r_mul(2.0f, r_add(r_mul(x, x), r_mul(y, y))));
    float s2[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) s2[a] = r_add(r_mul(rule_exp(r_mul(2.0f, ls[a])), 1.0001f), rho2);
    const int I[6] = {0, 0, 0, 1, 1, 2}, J[6] = {0, 1, 2, 1, 2, 2};
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        const int i = I[k], j = J[k];
        S[k] = r_add(r_add(r_mul(r_mul(R[3 * i], R[3 * j]), s2[0]), r_mul(r_mul(R[3 * i + 1], R[3 * j + 1]), s2[1])),
                     r_mul(r_mul(R[3 * i + 2], R[3 * j + 2]), s2[2]));
    }
}

// View part.  el (ELL_F floats), written when the test applies (returns true):
//   pinhole: the ellipse in pixels, Q(p) = (p - c)^T [[A,B],[B,C]] (p - c):
//            c_x c_y A B C, threshold 1.01 rhs, -B/C, -B/A;
//   fisheye: the ellipse in the plane tangent to the unit sphere at
//            u = (mu - o)/L (gnomonic coordinates in the basis e1, e2 = u x e1):
//            c_x c_y G00 G01 G11, sqrt(1.01 rhs), sqrt(tr G), e1 (3).
// g: scene record (kap ks kr r1sq s2); L: |mu - o|; m: the largest tile footprint bound.
static __device__ bool rule_ellipse(const CamParams &c, const float *g, float L, const float mu[3], const float S[6],
                                    float m, float el[ELL_F]) {
    const float kap = g[0], ks = g[1], kr = g[2], r1sq = g[3], s2 = g[4];
    const float sm = r_sqrt(m);
    const float cc = r_mul(kr, sm);
    const float rfc = r_mul(255.0f, ks);
    float tb, rf;
    if (cc < 1.0f) {
        const float tbf = r_div(r_add(L, ks), r_sub(1.0f, cc));
        const float rff = r_mul(kap, r_sqrt(r_add(s2, r_mul(r_mul(r_mul(tbf, tbf), r1sq), m))));
        rf = fminf(rff, rfc);
        tb = fminf(tbf, r_add(L, rf));
    } else {
        rf = rfc;
        tb = r_add(L, rf);
    }
    if (!(L > rf)) return false;
    const float w0 = r_sub(mu[0], c.o[0]), w1 = r_sub(mu[1], c.o[1]), w2 = r_sub(mu[2], c.o[2]);
    // frame F (columns, world): the camera axes (pinhole) or e1, e2, u (fisheye);
    // v = (mu - o)/L in that frame
    float F[9], v[3];
    if (c.model == 0) {
#pragma unroll
        for (int k = 0; k < 9; ++k) F[k] = c.R[k];
        const float iL = r_div(1.0f, L);
#pragma unroll
        for (int j = 0; j < 3; ++j)
            v[j] = r_mul(r_add(r_add(r_mul(c.R[j], w0), r_mul(c.R[3 + j], w1)), r_mul(c.R[6 + j], w2)), iL);
        if (!(v[2] > 0.0f && r_mul(v[2], v[2]) >= 0.05f)) return false;
    } else {
        const float u[3] = {r_div(w0, L), r_div(w1, L), r_div(w2, L)};
        const float au0 = fabsf(u[0]), au1 = fabsf(u[1]), au2 = fabsf(u[2]);
        const int k = (au0 <= au1 && au0 <= au2) ? 0 : (au1 <= au2 ? 1 : 2);
        float b[3] = {0.0f, 0.0f, 0.0f};
        b[k] = 1.0f;
        const float uk = u[k];
#pragma unroll
        for (int j = 0; j < 3; ++j) b[j] = r_sub(b[j], r_mul(uk, u[j]));
        const float nb = r_sqrt(r_add(r_add(r_mul(b[0], b[0]), r_mul(b[1], b[1])), r_mul(b[2], b[2])));
        const float e1[3] = {r_div(b[0], nb), r_div(b[1], nb), r_div(b[2], nb)};
        const float e2[3] = {r_sub(r_mul(u[1], e1[2]), r_mul(u[2], e1[1])),
                             r_sub(r_mul(u[2], e1[0]), r_mul(u[0], e1[2])),
                             r_sub(r_mul(u[0], e1[1]), r_mul(u[1], e1[0]))};
#pragma unroll
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
    // covariance in the frame: F^T Sigma F
    const float Sf[9] = {S[0], S[1], S[2], S[1], S[3], S[4], S[2], S[4], S[5]};
    float T[9];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int k = 0; k < 3; ++k)
            T[3 * i + k] = r_add(r_add(r_mul(Sf[3 * i], F[k]), r_mul(Sf[3 * i + 1], F[3 + k])),
                                 r_mul(Sf[3 * i + 2], F[6 + k]));
    float Cc[6];
    {
        const int I[6] = {0, 0, 0, 1, 1, 2}, J[6] = {0, 1, 2, 1, 2, 2};
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            const int j = I[k], l = J[k];
            Cc[k] = r_add(r_add(r_mul(F[j], T[l]), r_mul(F[3 + j], T[3 + l])), r_mul(F[6 + j], T[6 + l]));
        }
    }
    const float iso = r_add(r_mul(r_mul(tb, tb), m), r_mul(1e-5f, s2));
    Cc[0] = r_add(Cc[0], iso);
    Cc[3] = r_add(Cc[3], iso);
    Cc[5] = r_add(Cc[5], iso);
    const float tau = r_div(r_add(r_add(Cc[0], Cc[3]), Cc[5]), 3.0f);
    const float it = r_div(1.0f, tau);
    const float cxx = r_add(r_mul(Cc[0], it), 1e-4f), cxy = r_mul(Cc[1], it), cxz = r_mul(Cc[2], it);
    const float cyy = r_add(r_mul(Cc[3], it), 1e-4f), cyz = r_mul(Cc[4], it), czz = r_add(r_mul(Cc[5], it), 1e-4f);
    const float k2 = r_div(r_mul(r_mul(kap, kap), tau), r_mul(L, L));
    // inverse by the adjugate
    const float a00 = r_sub(r_mul(cyy, czz), r_mul(cyz, cyz));
    const float a01 = r_sub(r_mul(cxz, cyz), r_mul(cxy, czz));
    const float a02 = r_sub(r_mul(cxy, cyz), r_mul(cxz, cyy));
    const float a11 = r_sub(r_mul(cxx, czz), r_mul(cxz, cxz));
    const float a12 = r_sub(r_mul(cxy, cxz), r_mul(cxx, cyz));
    const float det = r_add(r_add(r_mul(cxx, a00), r_mul(cxy, a01)), r_mul(cxz, a02));
    if (!(det > 1e-12f)) return false;
    const float id = r_div(1.0f, det);
    const float i00 = r_mul(a00, id), i01 = r_mul(a01, id), i02 = r_mul(a02, id);
    const float i11 = r_mul(a11, id), i12 = r_mul(a12, id);
    const float i22 = r_mul(r_sub(r_mul(cxx, cyy), r_mul(cxy, cxy)), id);
    const float wx = r_add(r_add(r_mul(i00, v[0]), r_mul(i01, v[1])), r_mul(i02, v[2]));
    const float wy = r_add(r_add(r_mul(i01, v[0]), r_mul(i11, v[1])), r_mul(i12, v[2]));
    const float wz = r_add(r_add(r_mul(i02, v[0]), r_mul(i12, v[1])), r_mul(i22, v[2]));
    const float a = r_add(r_add(r_mul(v[0], wx), r_mul(v[1], wy)), r_mul(v[2], wz));
    const float am = r_sub(a, k2);
    if (!(am > r_mul(0.01f, k2))) return false;
    const float G00 = r_sub(r_mul(am, i00), r_mul(wx, wx));
    const float G01 = r_sub(r_mul(am, i01), r_mul(wx, wy));
    const float G11 = r_sub(r_mul(am, i11), r_mul(wy, wy));
    const float dG = r_sub(r_mul(G00, G11), r_mul(G01, G01));
    const float tG = r_add(G00, G11);
    if (!(G00 > 0.0f && dG > r_mul(1e-6f, r_mul(tG, tG)))) return false;
    const float ivz = r_div(1.0f, v[2]);
    const float hx = r_mul(r_mul(k2, wx), ivz), hy = r_mul(r_mul(k2, wy), ivz);
    const float k0 = r_mul(r_mul(k2, a), r_mul(ivz, ivz));
    const float idG = r_div(1.0f, dG);
    const float dcx = r_mul(r_sub(r_mul(G11, hx), r_mul(G01, hy)), idG);
    const float dcy = r_mul(r_sub(r_mul(G00, hy), r_mul(G01, hx)), idG);
    const float rhs = r_add(k0, r_add(r_mul(hx, dcx), r_mul(hy, dcy)));
    if (!(rhs > 0.0f && rhs < 1e30f)) return false;
    if (c.model == 0) {
        el[0] = r_add(r_mul(c.fx, r_add(r_mul(v[0], ivz), dcx)), c.cx);
        el[1] = r_add(r_mul(c.fy, r_add(r_mul(v[1], ivz), dcy)), c.cy);
        el[2] = r_div(G00, r_mul(c.fx, c.fx));
        el[3] = r_div(G01, r_mul(c.fx, c.fy));
        el[4] = r_div(G11, r_mul(c.fy, c.fy));
        el[5] = r_mul(rhs, 1.01f);
        el[6] = r_div(-el[3], el[4]);
        el[7] = r_div(-el[3], el[2]);
    } else {
        el[0] = dcx;
        el[1] = dcy;
        el[2] = G00;
        el[3] = G01;
        el[4] = G11;
        el[5] = r_sqrt(r_mul(rhs, 1.01f));
        el[6] = r_sqrt(tG);
    }
    return true;
}

// Fisheye tiles: the tile's rays lie within gamma of its axis a (sin(gamma/2) =
// t[3]), so along the arc from a their gnomonic images move at most
// gamma / cos^2(phi + gamma) (phi: the angle of a from u); with the G-norm
// below sqrt(tr G) times the Euclidean one, a tile reaching the ellipse has
// |p_a - c|_G <= sqrt(threshold) + sqrt(tr G) gamma / cos^2(phi + gamma), with
// gamma <= 2 sin(gamma/2) / cos(gamma/2).  Multiplied through by cos^2(phi) =
// (a.u)^2 (p_a = (a.e1, a.e2) / a.u), cos^4(phi + gamma) and cos^2(gamma/2), the
// test needs no division.  Tiles reaching beyond cos(phi + gamma) = 0.2 are kept.
template <int ST>
__device__ __forceinline__ bool kb_ellipse_test(const float *el, const float4 gv, const float *t) {
    const float ca = r_add(r_add(r_mul(t[0], gv.x), r_mul(t[1], gv.y)), r_mul(t[2], gv.z));
    const float s = t[3], ch = t[4];
    const float sp = r_sqrt(fmaxf(r_sub(1.0f, r_mul(ca, ca)), 0.0f));
    const float cg = r_sub(1.0f, r_mul(2.0f, r_mul(s, s)));
    const float sg = r_mul(2.0f, r_mul(s, ch));
    const float cpg = r_sub(r_mul(ca, cg), r_mul(sp, sg));
    if (!(cpg > 0.2f)) return true;
    const float e1x = el[7 * ST], e1y = el[8 * ST], e1z = el[9 * ST];
    const float e2x = r_sub(r_mul(gv.y, e1z), r_mul(gv.z, e1y));
    const float e2y = r_sub(r_mul(gv.z, e1x), r_mul(gv.x, e1z));
    const float e2z = r_sub(r_mul(gv.x, e1y), r_mul(gv.y, e1x));
    const float nx = r_sub(r_add(r_add(r_mul(t[0], e1x), r_mul(t[1], e1y)), r_mul(t[2], e1z)), r_mul(el[0], ca));
    const float ny = r_sub(r_add(r_add(r_mul(t[0], e2x), r_mul(t[1], e2y)), r_mul(t[2], e2z)), r_mul(el[ST], ca));
    const float Qn = r_add(r_mul(nx, r_add(r_mul(el[2 * ST], nx), r_mul(2.0f, r_mul(el[3 * ST], ny)))),
                           r_mul(el[4 * ST], r_mul(ny, ny)));
    const float c2 = r_mul(cpg, cpg);
    const float lhs = r_mul(r_mul(Qn, r_mul(c2, c2)), r_mul(ch, ch));
    const float r = r_add(r_mul(r_mul(el[5 * ST], c2), ch), r_mul(r_mul(2.0f, s), el[6 * ST]));
    return lhs <= r_mul(r_mul(r, r), r_mul(ca, ca));
}

// Tile (tx, ty) against an ellipse: the minimum over the tile's pixel-centre
// rectangle (grown by `grow` pixels) of Q(p) = (p - c)^T [[A,B],[B,C]] (p - c)
// is at most q.x.  With c outside the rectangle the minimum lies on an edge
// whose line separates c from it, at the clamped stationary point of Q along
// that edge.
__device__ __forceinline__ bool ellipse_rect_test(const CamParams &c, const float *e, const float4 q, int tx,
                                                  int ty, float grow) {
    const float x0 = r_sub((float)(TILE * tx) + 0.5f, grow), y0 = r_sub((float)(TILE * ty) + 0.5f, grow);
    const float x1 = r_add(fminf((float)(TILE * tx) + (float)TILE - 0.5f, (float)c.W - 0.5f), grow);
    const float y1 = r_add(fminf((float)(TILE * ty) + (float)TILE - 0.5f, (float)c.H - 0.5f), grow);
    const float dx0 = r_sub(x0, e[0]), dx1 = r_sub(x1, e[0]), dy0 = r_sub(y0, e[1]), dy1 = r_sub(y1, e[1]);
    const bool sx = dx0 > 0.0f || dx1 < 0.0f, sy = dy0 > 0.0f || dy1 < 0.0f;
    if (!sx && !sy) return true;
    float best = 3.0e38f;
    if (sx) {
        const float x = dx0 > 0.0f ? dx0 : dx1;
        const float y = fminf(fmaxf(r_mul(q.y, x), dy0), dy1);
        best = r_add(r_mul(x, r_add(r_mul(e[2], x), r_mul(2.0f, r_mul(e[3], y)))), r_mul(e[4], r_mul(y, y)));
    }
    if (sy) {
        const float y = dy0 > 0.0f ? dy0 : dy1;
        const float x = fminf(fmaxf(r_mul(q.z, y), dx0), dx1);
        best = fminf(best, r_add(r_mul(x, r_add(r_mul(e[2], x), r_mul(2.0f, r_mul(e[3], y)))),
                                 r_mul(e[4], r_mul(y, y))));
    }
    return best <= q.x;
}

constexpr float ELL_GROW = 0.05f;   // pixel-centre rectangle growth of the silhouette test

// The silhouette test of tile (tx, ty) with record t (its cone) for a slot whose
// ellipse applies; el[k * ST] is the record's k-th float, gv = (u, L) of the Gaussian.
template <int ST>
__device__ __forceinline__ bool ell_keep(const CamParams &c, const float *el, const float4 gv, const float *t, int tx,
                                         int ty) {
    if (c.model == 0) {
        const float e[5] = {el[0], el[ST], el[2 * ST], el[3 * ST], el[4 * ST]};
        return ellipse_rect_test(c, e, make_float4(el[5 * ST], el[6 * ST], el[7 * ST], 0.0f), tx, ty, ELL_GROW);
    }
    return kb_ellipse_test<ST>(el, gv, t);
}

}  // namespace conegs
