// Per pixel-Gaussian pair response (Sec. 4.1-4.2) in FP32 registers.
// Reciprocals, square roots and exp use the SFU approximations (about 1-2 ulp),
// far inside the 1e-4 output tolerance.
//
// With d_u = W d, g_i = W delta_i (W = W_eff), n = |d_u|^2:
//   t* = -<o_u, d_u>/n,  q = o_u + t* d_u                          (Eq. 2)
//   e_i = t* (g_i - d_u <d_u, g_i>/n) = t* M_perp W delta_i          (Eq. 6)
//   Sigma_fp = E E^T / 3, E = [e_x e_y]                               (Eq. 8)
// Eq. 12 keeps only the world-space footprint variance beyond rho^2.  The
// world half-edges are f_i = W^-1 e_i = t* (delta_i - d <d_u, g_i>/n); with
// H' = [f_i . f_j]/3 (eigenpairs lambda_j, v_j) the clamped, re-whitened
// footprint is E K E^T with K = sum_j max(lambda_j - rho^2, 0)/(3 lambda_j)
// v_j v_j^T, a 2x2 matrix function of H' (rho = 0 gives K = I/3).
// A = I + E K E^T, so with G = E^T E and b = E^T q (Sylvester / Woodbury):
//   det A = det(I + G K),  q^T A^-1 q = |q|^2 - b^T K (I + G K)^-1 b
//   T = sigma_eff det(A)^-1/2 exp(-q^T A^-1 q / 2)                   (Eq. 9)
// with q^T A^-1 q clamped below by |q|^2 / det A (exact bound, see below).
// No 3x3 matrix and no plane basis is formed.
#pragma once
#include "common.cuh"

namespace conegs {

struct PixelRays {
    float d[3], dx[3], dy[3];
    float d_dx, d_dy, dxdx, dxdy, dydy;   // for the marginal rule (Eq. 12)
};

// Intermediates of one pair evaluation, kept for the adjoint.
struct PairFwd {
    float du[3], gx[3], gy[3], inv_n, p, ts, q[3], qq, cx, cy, ex[3], ey[3];
    float G00, G01, G11, b0, b1;
    int kcase;                 // 0: K = I/3; 1: K = (I - rho2 H'^-1)/3; 2: rank-1 K; 3: K = 0
    float k00, k01, k11;
    float t2, A00, A01, A11, h00, h01, h11;
    float m00, m01, m10, m11, det, p00, p01, p10, p11, bPb, inv_det;
    bool clamped;              // Q = |q|^2/det (lower bound) was active
    float T;
};

__device__ __forceinline__ float dot3(const float a[3], const float b[3]) {
    return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}

// 2x2 matrix function K = f(H') of Eq. 12 (H' symmetric PSD), f(l) = max(l - rho2, 0) / (3 l).
// Returns the case (1: both eigenvalues above rho2, 2: only the larger, 3: neither).
__device__ __forceinline__ int marginal_K(float h00, float h01, float h11, float rho2, float &k00, float &k01,
                                          float &k11) {
    const float mean = 0.5f * (h00 + h11);
    const float half = 0.5f * (h00 - h11);
    const float r2 = half * half + h01 * h01;
    const float rad = r2 > 0.0f ? r2 * rsqrtf(r2) : 0.0f;
    const float l1 = mean + rad;
    if (!(l1 > rho2)) {
        k00 = k01 = k11 = 0.0f;
        return 3;
    }
    const float det = h00 * h11 - h01 * h01;
    const float l2 = __fdividef(fmaxf(det, 0.0f), l1);   // smaller eigenvalue without cancellation
    if (l2 > rho2) {
        // both directions exceed the floor: K = (I - rho2 H'^-1)/3
        const float s = __fdividef(rho2, det);
        k00 = (1.0f - s * h11) * (1.0f / 3.0f);
        k11 = (1.0f - s * h00) * (1.0f / 3.0f);
        k01 = (s * h01) * (1.0f / 3.0f);
        return 1;
    } else {
        // only the major direction exceeds: K = f(l1) (H' - l2 I)/(l1 - l2)
        const float sc = __fdividef(l1 - rho2, 3.0f * l1 * (l1 - l2));
        k00 = sc * (h00 - l2);
        k11 = sc * (h11 - l2);
        k01 = sc * h01;
        return 2;
    }
}

// Response of one pair.  r0..r2 = [W row | o_u], sig = sigma_eff, rho2.
// Returns false when t* <= T_NEAR (pair skipped).  With STORE the
// intermediates are copied to *st (the arithmetic is the same either way).
template <bool FILTER, bool STORE = false>
__device__ __forceinline__ bool pair_response(const float4 r0, const float4 r1, const float4 r2, const float sig,
                                              const float rho2, const bool additive, const PixelRays &px,
                                              float &T, PairFwd *st = nullptr) {
    const float du0 = r0.x * px.d[0] + r0.y * px.d[1] + r0.z * px.d[2];
    const float du1 = r1.x * px.d[0] + r1.y * px.d[1] + r1.z * px.d[2];
    const float du2 = r2.x * px.d[0] + r2.y * px.d[1] + r2.z * px.d[2];
    const float n = du0 * du0 + du1 * du1 + du2 * du2;
    const float inv_n = __fdividef(1.0f, n);
    const float p = r0.w * du0 + r1.w * du1 + r2.w * du2;
    const float ts = -p * inv_n;
    if (!(ts > T_NEAR)) return false;
    const float q0 = r0.w + ts * du0, q1 = r1.w + ts * du1, q2 = r2.w + ts * du2;
    const float qq = q0 * q0 + q1 * q1 + q2 * q2;
    if (STORE) {
        st->du[0] = du0; st->du[1] = du1; st->du[2] = du2;
        st->inv_n = inv_n; st->p = p; st->ts = ts;
        st->q[0] = q0; st->q[1] = q1; st->q[2] = q2; st->qq = qq;
    }
    if (!FILTER) {
        T = sig * __expf(-0.5f * qq);
        if (STORE) st->T = T;
        return true;
    }
    const float gx0 = r0.x * px.dx[0] + r0.y * px.dx[1] + r0.z * px.dx[2];
    const float gx1 = r1.x * px.dx[0] + r1.y * px.dx[1] + r1.z * px.dx[2];
    const float gx2 = r2.x * px.dx[0] + r2.y * px.dx[1] + r2.z * px.dx[2];
    const float gy0 = r0.x * px.dy[0] + r0.y * px.dy[1] + r0.z * px.dy[2];
    const float gy1 = r1.x * px.dy[0] + r1.y * px.dy[1] + r1.z * px.dy[2];
    const float gy2 = r2.x * px.dy[0] + r2.y * px.dy[1] + r2.z * px.dy[2];
    const float cx = (du0 * gx0 + du1 * gx1 + du2 * gx2) * inv_n;
    const float cy = (du0 * gy0 + du1 * gy1 + du2 * gy2) * inv_n;
    const float ex0 = ts * (gx0 - cx * du0), ex1 = ts * (gx1 - cx * du1), ex2 = ts * (gx2 - cx * du2);
    const float ey0 = ts * (gy0 - cy * du0), ey1 = ts * (gy1 - cy * du1), ey2 = ts * (gy2 - cy * du2);
    const float G00 = ex0 * ex0 + ex1 * ex1 + ex2 * ex2;
    const float G01 = ex0 * ey0 + ex1 * ey1 + ex2 * ey2;
    const float G11 = ey0 * ey0 + ey1 * ey1 + ey2 * ey2;
    const float b0 = ex0 * q0 + ex1 * q1 + ex2 * q2;
    const float b1 = ey0 * q0 + ey1 * q1 + ey2 * q2;
    float det, bPb;
    if (rho2 == 0.0f || additive) {
        // K = I/3
        const float m00 = 1.0f + G00 * (1.0f / 3.0f), m11 = 1.0f + G11 * (1.0f / 3.0f), m01 = G01 * (1.0f / 3.0f);
        det = m00 * m11 - m01 * m01;
        bPb = (b0 * b0 * m11 - 2.0f * b0 * b1 * m01 + b1 * b1 * m00) * (1.0f / 3.0f);
        if (STORE) {
            st->kcase = 0;
            st->k00 = st->k11 = 1.0f / 3.0f; st->k01 = 0.0f;
            st->m00 = m00; st->m01 = m01; st->m10 = m01; st->m11 = m11;
            st->p00 = m11 * (1.0f / 3.0f); st->p01 = -m01 * (1.0f / 3.0f);
            st->p10 = -m01 * (1.0f / 3.0f); st->p11 = m00 * (1.0f / 3.0f);
        }
    } else {
        const float t2 = ts * ts * (1.0f / 3.0f);
        const float A00 = px.dxdx - 2.0f * cx * px.d_dx + cx * cx;
        const float A01 = px.dxdy - cx * px.d_dy - cy * px.d_dx + cx * cy;
        const float A11 = px.dydy - 2.0f * cy * px.d_dy + cy * cy;
        const float h00 = t2 * A00, h01 = t2 * A01, h11 = t2 * A11;
        float k00, k01, k11;
        const int kc = marginal_K(h00, h01, h11, rho2, k00, k01, k11);
        const float m00 = 1.0f + G00 * k00 + G01 * k01, m01 = G00 * k01 + G01 * k11;
        const float m10 = G01 * k00 + G11 * k01, m11 = 1.0f + G01 * k01 + G11 * k11;
        det = m00 * m11 - m01 * m10;
        const float p00 = k00 * m11 - k01 * m10, p01 = k01 * m00 - k00 * m01;
        const float p10 = k01 * m11 - k11 * m10, p11 = k11 * m00 - k01 * m01;
        bPb = b0 * b0 * p00 + b0 * b1 * (p01 + p10) + b1 * b1 * p11;
        if (STORE) {
            st->kcase = kc;
            st->k00 = k00; st->k01 = k01; st->k11 = k11;
            st->t2 = t2; st->A00 = A00; st->A01 = A01; st->A11 = A11;
            st->h00 = h00; st->h01 = h01; st->h11 = h11;
            st->m00 = m00; st->m01 = m01; st->m10 = m10; st->m11 = m11;
            st->p00 = p00; st->p01 = p01; st->p10 = p10; st->p11 = p11;
        }
    }
    // q^T A^-1 q >= |q|^2 / lambda_max(A) >= |q|^2 / det A (A = I + a PSD rank-2
    // matrix), a bound that also guards the FP32 difference against cancellation
    // for far, flat Gaussians seen at grazing angles.
    const float rdet = rsqrtf(det);
    const float inv_det = rdet * rdet;
    const float Qa = qq - bPb * inv_det, Qb = qq * inv_det;
    const float Q = fmaxf(Qa, Qb);
    T = sig * rdet * __expf(-0.5f * Q);
    if (STORE) {
        st->gx[0] = gx0; st->gx[1] = gx1; st->gx[2] = gx2;
        st->gy[0] = gy0; st->gy[1] = gy1; st->gy[2] = gy2;
        st->cx = cx; st->cy = cy;
        st->ex[0] = ex0; st->ex[1] = ex1; st->ex[2] = ex2;
        st->ey[0] = ey0; st->ey[1] = ey1; st->ey[2] = ey2;
        st->G00 = G00; st->G01 = G01; st->G11 = G11; st->b0 = b0; st->b1 = b1;
        st->det = det; st->bPb = bPb; st->inv_det = inv_det;
        st->clamped = !(Qa >= Qb);
        st->T = T;
    }
    return true;
}

}  // namespace conegs
