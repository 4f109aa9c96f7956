// Device-side central-camera model shared by the ray table (K1) and the
// training-floor kernel (Eq. 11): FP32 validity rule, Kannala-Brandt
// inversion and cancellation-free half-pixel differentials.
#pragma once
#include "common.cuh"

namespace conegs {


// Pixel validity (the FP32 rule; the same decision everywhere the library
// needs it: ray table, binning, floor).
__device__ __forceinline__ bool valid_xy(const CamParams &c, float x, float y) {
    if (c.model == 0) return true;
    float a = __fdiv_rn(__fsub_rn(x, c.cx), c.fx);
    float b = __fdiv_rn(__fsub_rn(y, c.cy), c.fy);
    float r2 = __fadd_rn(__fmul_rn(a, a), __fmul_rn(b, b));
    return r2 <= c.rlim2;
}

__device__ __forceinline__ float kb_P(const CamParams &c, float th) {
    float t2 = th * th;
    return th * (1.0f + t2 * (c.k[0] + t2 * (c.k[1] + t2 * (c.k[2] + t2 * c.k[3]))));
}
__device__ __forceinline__ float kb_dP(const CamParams &c, float th) {
    float t2 = th * th;
    return 1.0f + t2 * (3.0f * c.k[0] + t2 * (5.0f * c.k[1] + t2 * (7.0f * c.k[2] + t2 * 9.0f * c.k[3])));
}
__device__ __forceinline__ double kb_Pd(const CamParams &c, double th) {
    double t2 = th * th;
    return th * (1.0 + t2 * ((double)c.k[0] + t2 * ((double)c.k[1] + t2 * ((double)c.k[2] + t2 * (double)c.k[3]))));
}
__device__ __forceinline__ double kb_dPd(const CamParams &c, double th) {
    double t2 = th * th;
    return 1.0 + t2 * (3.0 * c.k[0] + t2 * (5.0 * c.k[1] + t2 * (7.0 * c.k[2] + t2 * 9.0 * (double)c.k[3])));
}

constexpr float KB_FP64_THETA = 1.2f;  // polish in FP64 beyond ~69 deg

// theta with theta_d(theta) = r, theta in [0, theta_lim].
static __device__ float kb_theta(const CamParams &c, float r) {
    float th = fminf(r, c.thlim);
    for (int it = 0; it < 10; ++it) {
        float step = (kb_P(c, th) - r) / kb_dP(c, th);
        th = fminf(fmaxf(th - step, 0.0f), c.thlim);
    }
    if (th > KB_FP64_THETA) {
        double t = th;
        for (int it = 0; it < 2; ++it) {
            double fp = kb_dPd(c, t);
            if (fp > 0.0) t -= (kb_Pd(c, t) - (double)r) / fp;
        }
        t = fmin(fmax(t, 0.0), (double)c.thlim);
        th = (float)t;
    }
    return th;
}

// Increment Delta with theta_d(th + Delta) - theta_d(th) = dr, from the
// divided differences S_n = ((th+D)^n - th^n)/D (all terms positive, no
// cancellation): S_1 = 1, S_{n+2} = u^2 S_n + th^n (u + th), u = th + D.
template <typename T>
__device__ __forceinline__ T kb_dtheta_t(const CamParams &c, T th, T dr) {
    T k0 = c.k[0], k1 = c.k[1], k2 = c.k[2], k3 = c.k[3];
    T t2 = th * th;
    T dP0 = T(1) + t2 * (T(3) * k0 + t2 * (T(5) * k1 + t2 * (T(7) * k2 + t2 * T(9) * k3)));
    T D = dr / dP0;
    for (int it = 0; it < 3; ++it) {
        T u = th + D, u2 = u * u, w = u + th;
        T th3 = t2 * th, th5 = th3 * t2, th7 = th5 * t2;
        T S3 = u2 + th * w;
        T S5 = u2 * S3 + th3 * w;
        T S7 = u2 * S5 + th5 * w;
        T S9 = u2 * S7 + th7 * w;
        T Q = T(1) + k0 * S3 + k1 * S5 + k2 * S7 + k3 * S9;
        T F = D * Q - dr;
        T dP = T(1) + u2 * (T(3) * k0 + u2 * (T(5) * k1 + u2 * (T(7) * k2 + u2 * T(9) * k3)));
        D -= F / dP;
    }
    return D;
}

// One KB edge differential (camera frame) for normalised offset h along axis.
static __device__ void kb_edge(const CamParams &c, float a, float b, float r, float th, float sth, float g, int axis,
                        float h, float out[3]) {
    float ae = axis == 0 ? a + h : a;
    float be = axis == 1 ? b + h : b;
    float re = sqrtf(ae * ae + be * be);
    float along = axis == 0 ? a : b;
    float dr = h * (2.0f * along + h) / (re + r);          // r' - r without cancellation
    float D = th > KB_FP64_THETA ? (float)kb_dtheta_t<double>(c, (double)th, (double)dr)
                                 : kb_dtheta_t<float>(c, th, dr);
    float s_half = sinf(0.5f * D);
    float sh, ch;
    sincosf(th + 0.5f * D, &sh, &ch);
    float dcos = -2.0f * sh * s_half;                        // cos(th+D) - cos(th)
    float ge = re > 1e-30f ? sinf(th + D) / re : 1.0f;
    float dg;                                                // g' - g, g = sin(theta)/r
    if (r > 1e-30f && re > 1e-30f)
        dg = 2.0f * ch * s_half / re - sth * dr / (r * re);
    else
        dg = ge - g;
    if (axis == 0) {
        out[0] = ge * h + dg * a;
        out[1] = dg * b;
    } else {
        out[0] = dg * a;
        out[1] = ge * h + dg * b;
    }
    out[2] = dcos;
}

__device__ __forceinline__ void rotate(const CamParams &c, const float v[3], float w[3]) {
#pragma unroll
    for (int i = 0; i < 3; ++i) w[i] = c.R[3 * i] * v[0] + c.R[3 * i + 1] * v[1] + c.R[3 * i + 2] * v[2];
}


// Camera-frame centre ray and half-pixel differentials of image point (x, y)
// (forward differences, or backward ones where the forward edge point leaves
// the valid disc).  Returns false outside the valid domain.
__device__ __forceinline__ bool point_rays(const CamParams &c, float x, float y, float vd[3], float vx[3],
                                           float vy[3]) {
    vd[0] = vd[1] = vd[2] = vx[0] = vx[1] = vx[2] = vy[0] = vy[1] = vy[2] = 0.0f;
    bool ok = valid_xy(c, x, y);
    if (ok) {
        const float a = (x - c.cx) / c.fx, b = (y - c.cy) / c.fy;
        if (c.model == 0) {
            const float n2 = a * a + b * b + 1.0f, sn = sqrtf(n2), inv = 1.0f / sn;
            vd[0] = a * inv; vd[1] = b * inv; vd[2] = inv;
            const float hx = 0.5f / c.fx, hy = 0.5f / c.fy;
            {
                const float nx2 = n2 + hx * (2.0f * a + hx), snx = sqrtf(nx2), invx = 1.0f / snx;
                const float dinv = -hx * (2.0f * a + hx) * inv * invx / (sn + snx);
                vx[0] = hx * invx + a * dinv; vx[1] = b * dinv; vx[2] = dinv;
            }
            {
                const float ny2 = n2 + hy * (2.0f * b + hy), sny = sqrtf(ny2), invy = 1.0f / sny;
                const float dinv = -hy * (2.0f * b + hy) * inv * invy / (sn + sny);
                vy[0] = a * dinv; vy[1] = hy * invy + b * dinv; vy[2] = dinv;
            }
        } else {
            const float r = sqrtf(a * a + b * b);
            const float th = kb_theta(c, r);
            float sth, cth;
            sincosf(th, &sth, &cth);
            const float g = r > 1e-30f ? sth / r : 1.0f;
            vd[0] = g * a; vd[1] = g * b; vd[2] = cth;
            // forward difference unless the edge point leaves the valid disc
            const bool fx_ok = valid_xy(c, x + 0.5f, y), fy_ok = valid_xy(c, x, y + 0.5f);
            const float hx = (fx_ok ? 0.5f : -0.5f) / c.fx, hy = (fy_ok ? 0.5f : -0.5f) / c.fy;
            kb_edge(c, a, b, r, th, sth, g, 0, hx, vx);
            kb_edge(c, a, b, r, th, sth, g, 1, hy, vy);
            if (!fx_ok) { vx[0] = -vx[0]; vx[1] = -vx[1]; vx[2] = -vx[2]; }
            if (!fy_ok) { vy[0] = -vy[0]; vy[1] = -vy[1]; vy[2] = -vy[2]; }
        }
    }
    return ok;
}

}  // namespace conegs
