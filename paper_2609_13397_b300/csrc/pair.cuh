// Per pixel-Gaussian pair response (Sec. 4.1-4.2) in registers.
//
// The arithmetic type R is float for every Gaussian but the near-degenerate
// flat ones (effective scale ratio above FLAT_RATIO), which take R = double:
// their whitening W has a row of length 1/s_min, so the whitened camera
// centre o_u and ray d_u are large, t* and q = o_u + t* d_u cancel, and the
// final |q|^2 - b^T K (I + GK)^-1 b cancels again.  In FP32 the response of
// such a disk seen at a grazing angle is off by ~3e-4 at s_max/s_min = 300
// and by ~2e-3 at 10^4 (face-on); up to 100 it stays within ~5e-5, hence the
// threshold.  FP32 uses the SFU
// approximations of reciprocal, square root and exp (about 1-2 ulp), far
// inside the 1e-4 output tolerance; FP64 uses the correctly rounded ones.
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

// A Gaussian is "flat" (evaluated in FP64) when s_eff,max / s_eff,min > FLAT_RATIO
// (the effective scales of Eq. 10, after the floor).
constexpr float FLAT_RATIO = 100.0f;

struct PixelRays {
    float d[3], dx[3], dy[3];
    float d_dx, d_dy, dxdx, dxdy, dydy;   // for the marginal rule (Eq. 12)
};

// Intermediates of one pair evaluation, kept for the adjoint.
template <typename R>
struct PairFwdT {
    R du[3], gx[3], gy[3], inv_n, p, ts, q[3], qq, cx, cy, ex[3], ey[3];
    R G00, G01, G11, b0, b1;
    int kcase;                 // 0: K = I/3; 1: K = (I - rho2 H'^-1)/3; 2: rank-1 K; 3: K = 0
    R k00, k01, k11;
    R t2, A00, A01, A11, h00, h01, h11;
    R m00, m01, m10, m11, det, p00, p01, p10, p11, bPb, inv_det;
    bool clamped;              // Q = |q|^2/det (lower bound) was active
    R T;
};
using PairFwd = PairFwdT<float>;

// Elementary operations per arithmetic type.
template <typename R>
struct Ar;
template <>
struct Ar<float> {
    static __device__ __forceinline__ float div(float a, float b) { return __fdividef(a, b); }
    static __device__ __forceinline__ float rsqrt(float x) { return rsqrtf(x); }
    static __device__ __forceinline__ float sqrt(float x) { return sqrtf(x); }
    static __device__ __forceinline__ float exp(float x) { return __expf(x); }
    static __device__ __forceinline__ float max(float a, float b) { return fmaxf(a, b); }
};
template <>
struct Ar<double> {
    static __device__ __forceinline__ double div(double a, double b) { return a / b; }
    static __device__ __forceinline__ double rsqrt(double x) { return ::rsqrt(x); }
    static __device__ __forceinline__ double sqrt(double x) { return ::sqrt(x); }
    static __device__ __forceinline__ double exp(double x) { return ::exp(x); }
    static __device__ __forceinline__ double max(double a, double b) { return fmax(a, b); }
};

__device__ __forceinline__ float dot3(const float a[3], const float b[3]) {
    return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}

// Everything of a Gaussian's view record the response needs, in type R:
// W_eff rows, o_u, sigma_eff, rho^2.
template <typename R>
struct GaussRec {
    R W[9], ou[3], sig, rho2;
};

// The flat flag is the sign bit of the record's rho^2 word; a flat record keeps
// the low-order parts of o_u (o_u = hi + lo in FP64) in the three words after it.
__device__ __forceinline__ bool rec_is_flat(const float rho2_word) { return signbit(rho2_word); }
__device__ __forceinline__ bool rec_is_flat(const float4 r7) { return rec_is_flat(r7.x); }

__device__ __forceinline__ GaussRec<float> rec_f32(const float4 r0, const float4 r1, const float4 r2, float sig,
                                                   float rho2) {
    return GaussRec<float>{{r0.x, r0.y, r0.z, r1.x, r1.y, r1.z, r2.x, r2.y, r2.z}, {r0.w, r1.w, r2.w}, sig, rho2};
}

__device__ __forceinline__ GaussRec<double> rec_f64(const float4 r0, const float4 r1, const float4 r2, float sig,
                                                    const float4 r7) {
    return GaussRec<double>{{r0.x, r0.y, r0.z, r1.x, r1.y, r1.z, r2.x, r2.y, r2.z},
                            {(double)r0.w + (double)r7.y, (double)r1.w + (double)r7.z, (double)r2.w + (double)r7.w},
                            sig, (double)fabsf(r7.x)};
}

// 2x2 matrix function K = f(H') of Eq. 12 (H' symmetric PSD), f(l) = max(l - rho2, 0) / (3 l).
// Returns the case (1: both eigenvalues above rho2, 2: only the larger, 3: neither).
template <typename R>
__device__ __forceinline__ int marginal_K(R h00, R h01, R h11, R rho2, R &k00, R &k01, R &k11) {
    using A = Ar<R>;
    const R third = R(1) / R(3);
    const R mean = R(0.5) * (h00 + h11);
    const R half = R(0.5) * (h00 - h11);
    const R r2 = half * half + h01 * h01;
    const R rad = r2 > R(0) ? r2 * A::rsqrt(r2) : R(0);
    const R l1 = mean + rad;
    if (!(l1 > rho2)) {
        k00 = k01 = k11 = R(0);
        return 3;
    }
    const R det = h00 * h11 - h01 * h01;
    const R l2 = A::div(A::max(det, R(0)), l1);   // smaller eigenvalue without cancellation
    if (l2 > rho2) {
        // both directions exceed the floor: K = (I - rho2 H'^-1)/3
        const R s = A::div(rho2, det);
        k00 = (R(1) - s * h11) * third;
        k11 = (R(1) - s * h00) * third;
        k01 = (s * h01) * third;
        return 1;
    } else {
        // only the major direction exceeds: K = f(l1) (H' - l2 I)/(l1 - l2)
        const R sc = A::div(l1 - rho2, R(3) * l1 * (l1 - l2));
        k00 = sc * (h00 - l2);
        k11 = sc * (h11 - l2);
        k01 = sc * h01;
        return 2;
    }
}

// Response of one pair in arithmetic type R (the pixel's rays are FP32 and
// are widened for R = double).  Returns false when t* <= T_NEAR (pair
// skipped).  With STORE the intermediates are copied to *st (the arithmetic
// is the same either way).
template <bool FILTER, bool STORE = false, typename R = float>
__device__ __forceinline__ bool pair_response(const GaussRec<R> &g, const bool additive, const PixelRays &px,
                                              float &Tout, PairFwdT<R> *st = nullptr) {
    using A = Ar<R>;
    const R third = R(1) / R(3);
    const R *W = g.W;
    const R d0 = px.d[0], d1 = px.d[1], d2 = px.d[2];
    const R du0 = W[0] * d0 + W[1] * d1 + W[2] * d2;
    const R du1 = W[3] * d0 + W[4] * d1 + W[5] * d2;
    const R du2 = W[6] * d0 + W[7] * d1 + W[8] * d2;
    const R n = du0 * du0 + du1 * du1 + du2 * du2;
    const R inv_n = A::div(R(1), n);
    const R p = g.ou[0] * du0 + g.ou[1] * du1 + g.ou[2] * du2;
    const R ts = -p * inv_n;
    if (!(ts > R(T_NEAR))) return false;
    const R q0 = g.ou[0] + ts * du0, q1 = g.ou[1] + ts * du1, q2 = g.ou[2] + ts * du2;
    const R qq = q0 * q0 + q1 * q1 + q2 * q2;
    if (STORE) {
        st->du[0] = du0; st->du[1] = du1; st->du[2] = du2;
        st->inv_n = inv_n; st->p = p; st->ts = ts;
        st->q[0] = q0; st->q[1] = q1; st->q[2] = q2; st->qq = qq;
    }
    if (!FILTER) {
        const R T = g.sig * A::exp(R(-0.5) * qq);
        Tout = (float)T;
        if (STORE) st->T = T;
        return true;
    }
    const R x0 = px.dx[0], x1 = px.dx[1], x2 = px.dx[2];
    const R y0 = px.dy[0], y1 = px.dy[1], y2 = px.dy[2];
    const R gx0 = W[0] * x0 + W[1] * x1 + W[2] * x2;
    const R gx1 = W[3] * x0 + W[4] * x1 + W[5] * x2;
    const R gx2 = W[6] * x0 + W[7] * x1 + W[8] * x2;
    const R gy0 = W[0] * y0 + W[1] * y1 + W[2] * y2;
    const R gy1 = W[3] * y0 + W[4] * y1 + W[5] * y2;
    const R gy2 = W[6] * y0 + W[7] * y1 + W[8] * y2;
    const R cx = (du0 * gx0 + du1 * gx1 + du2 * gx2) * inv_n;
    const R cy = (du0 * gy0 + du1 * gy1 + du2 * gy2) * inv_n;
    const R ex0 = ts * (gx0 - cx * du0), ex1 = ts * (gx1 - cx * du1), ex2 = ts * (gx2 - cx * du2);
    const R ey0 = ts * (gy0 - cy * du0), ey1 = ts * (gy1 - cy * du1), ey2 = ts * (gy2 - cy * du2);
    const R G00 = ex0 * ex0 + ex1 * ex1 + ex2 * ex2;
    const R G01 = ex0 * ey0 + ex1 * ey1 + ex2 * ey2;
    const R G11 = ey0 * ey0 + ey1 * ey1 + ey2 * ey2;
    const R b0 = ex0 * q0 + ex1 * q1 + ex2 * q2;
    const R b1 = ey0 * q0 + ey1 * q1 + ey2 * q2;
    R det, bPb;
    if (g.rho2 == R(0) || additive) {
        // K = I/3
        const R m00 = R(1) + G00 * third, m11 = R(1) + G11 * third, m01 = G01 * third;
        det = m00 * m11 - m01 * m01;
        bPb = (b0 * b0 * m11 - R(2) * b0 * b1 * m01 + b1 * b1 * m00) * third;
        if (STORE) {
            st->kcase = 0;
            st->k00 = st->k11 = third; st->k01 = R(0);
            st->m00 = m00; st->m01 = m01; st->m10 = m01; st->m11 = m11;
            st->p00 = m11 * third; st->p01 = -m01 * third;
            st->p10 = -m01 * third; st->p11 = m00 * third;
        }
    } else {
        // the pixel's ray Gram terms: precomputed in FP32, recomputed for FP64
        R d_dx, d_dy, dxdx, dxdy, dydy;
        if (sizeof(R) == sizeof(float)) {
            d_dx = px.d_dx; d_dy = px.d_dy; dxdx = px.dxdx; dxdy = px.dxdy; dydy = px.dydy;
        } else {
            d_dx = d0 * x0 + d1 * x1 + d2 * x2;
            d_dy = d0 * y0 + d1 * y1 + d2 * y2;
            dxdx = x0 * x0 + x1 * x1 + x2 * x2;
            dxdy = x0 * y0 + x1 * y1 + x2 * y2;
            dydy = y0 * y0 + y1 * y1 + y2 * y2;
        }
        const R t2 = ts * ts * third;
        const R A00 = dxdx - R(2) * cx * d_dx + cx * cx;
        const R A01 = dxdy - cx * d_dy - cy * d_dx + cx * cy;
        const R A11 = dydy - R(2) * cy * d_dy + cy * cy;
        const R h00 = t2 * A00, h01 = t2 * A01, h11 = t2 * A11;
        R k00, k01, k11;
        const int kc = marginal_K<R>(h00, h01, h11, g.rho2, k00, k01, k11);
        const R m00 = R(1) + G00 * k00 + G01 * k01, m01 = G00 * k01 + G01 * k11;
        const R m10 = G01 * k00 + G11 * k01, m11 = R(1) + G01 * k01 + G11 * k11;
        det = m00 * m11 - m01 * m10;
        const R p00 = k00 * m11 - k01 * m10, p01 = k01 * m00 - k00 * m01;
        const R p10 = k01 * m11 - k11 * m10, p11 = k11 * m00 - k01 * m01;
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
    // for far Gaussians seen at grazing angles.
    const R rdet = A::rsqrt(det);
    const R inv_det = rdet * rdet;
    const R Qa = qq - bPb * inv_det, Qb = qq * inv_det;
    const R Q = A::max(Qa, Qb);
    const R T = g.sig * rdet * A::exp(R(-0.5) * Q);
    Tout = (float)T;
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
