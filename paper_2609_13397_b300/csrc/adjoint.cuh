// Reverse mode of the pair response (pair.cuh), written by hand.
#pragma once
#include "pair.cuh"

namespace conegs {

// Reverse-mode of pair_response<FILTER, true, R> given dL/dT, in the same
// arithmetic type R (divisions as products with Ops<R>::rcp: the SFU
// reciprocal in FP32, the correctly rounded one in FP64).  Accumulates dL/dW
// (9, row-major), dL/do_u (3) and returns dL/dsigma_eff.
template <bool FILTER, typename R>
__device__ __forceinline__ float pair_adjoint(const PairFwdT<R> &f, const GaussRec<R> &gr, const PixelRaysT<R> &px,
                                              float gT_in, float gW[9], float gou[3]) {
    using O = Ops<R>;
    const R third = R(1) / R(3);
    const R gT = gT_in, sig = gr.sig, rho2 = gr.rho2;
    const R T = f.T;
    const R gsig = sig > R(0) ? gT * T * O::rcp(sig) : R(0);
    const R gQ = R(-0.5) * T * gT;
    R gqq = R(0), gdu[3] = {R(0), R(0), R(0)}, gq[3] = {R(0), R(0), R(0)}, gts = R(0), ginv_n = R(0);
    R ggx[3] = {R(0), R(0), R(0)}, ggy[3] = {R(0), R(0), R(0)};
    R gou_r[3] = {R(0), R(0), R(0)};
    if (!FILTER) {
        gqq = gQ;
    } else {
        R gdet = -R(0.5) * T * gT * f.inv_det;             // T ~ det^-1/2
        R gbPb = R(0);
        if (!f.clamped) {                                    // Q = qq - bPb/det
            gqq = gQ;
            gbPb = -gQ * f.inv_det;
            gdet += gQ * f.bPb * f.inv_det * f.inv_det;
        } else {                                             // Q = qq/det
            gqq = gQ * f.inv_det;
            gdet += -gQ * f.qq * f.inv_det * f.inv_det;
        }
        // bPb = b0^2 p00 + b0 b1 (p01 + p10) + b1^2 p11
        const R b0 = f.b0, b1 = f.b1;
        const R gb0 = gbPb * (R(2) * b0 * f.p00 + b1 * (f.p01 + f.p10));
        const R gb1 = gbPb * (b0 * (f.p01 + f.p10) + R(2) * b1 * f.p11);
        const R gp00 = gbPb * b0 * b0, gp01 = gbPb * b0 * b1, gp10 = gp01, gp11 = gbPb * b1 * b1;
        // P = K adj(M)
        const R k00 = f.k00, k01 = f.k01, k11 = f.k11;
        const R m00 = f.m00, m01 = f.m01, m10 = f.m10, m11 = f.m11;
        R gk00 = gp00 * m11 - gp01 * m01;
        R gk01 = -gp00 * m10 + gp01 * m00 + gp10 * m11 - gp11 * m01;
        R gk11 = -gp10 * m10 + gp11 * m00;
        R gm00 = gp01 * k01 + gp11 * k11 + gdet * m11;
        R gm11 = gp00 * k00 + gp10 * k01 + gdet * m00;
        R gm01 = -gp01 * k00 - gp11 * k01 - gdet * m10;
        R gm10 = -gp00 * k01 - gp10 * k11 - gdet * m01;
        // M = I + G K
        const R G00 = f.G00, G01 = f.G01, G11 = f.G11;
        const R gG00 = gm00 * k00 + gm01 * k01;
        const R gG01 = gm00 * k01 + gm01 * k11 + gm10 * k00 + gm11 * k01;
        const R gG11 = gm10 * k01 + gm11 * k11;
        gk00 += gm00 * G00 + gm10 * G01;
        gk01 += gm00 * G01 + gm01 * G00 + gm10 * G11 + gm11 * G01;
        gk11 += gm01 * G01 + gm11 * G11;
        // K = f(H') (Eq. 12); H' = t2 A, t2 = ts^2/3
        R gcx = R(0), gcy = R(0);
        if (f.kcase == 1 || f.kcase == 2) {
            const R h00 = f.h00, h01 = f.h01, h11 = f.h11;
            R gh00 = R(0), gh01 = R(0), gh11 = R(0);
            const R dh = h00 * h11 - h01 * h01;
            if (f.kcase == 1) {                              // K = (I - rho2 H'^-1)/3
                const R inv_dh = O::rcp(dh);
                const R s = rho2 * inv_dh;
                const R gs = (-gk00 * h11 - gk11 * h00 + gk01 * h01) * third;
                gh11 += -gk00 * s * third;
                gh00 += -gk11 * s * third;
                gh01 += gk01 * s * third;
                const R gdh = -gs * s * inv_dh;
                gh00 += gdh * h11;
                gh11 += gdh * h00;
                gh01 += -R(2) * gdh * h01;
            } else {                                         // K = sc (H' - l2 I)
                const R mean = R(0.5) * (h00 + h11), half = R(0.5) * (h00 - h11);
                const R r2 = half * half + h01 * h01;
                const R rad = O::root(r2);
                const R l1 = mean + rad;
                const R inv_l1 = O::rcp(l1);
                const R l2 = O::max(dh, R(0)) * inv_l1;
                const R D = R(3) * l1 * (l1 - l2);
                const R inv_D = O::rcp(D);
                const R sc = (l1 - rho2) * inv_D;
                const R gsc = gk00 * (h00 - l2) + gk11 * (h11 - l2) + gk01 * h01;
                gh00 += gk00 * sc;
                gh11 += gk11 * sc;
                gh01 += gk01 * sc;
                R gl2 = -(gk00 + gk11) * sc;
                const R gN = gsc * inv_D, gD = -gsc * sc * inv_D;
                R gl1 = gN + gD * R(3) * (R(2) * l1 - l2);
                gl2 += gD * (-R(3) * l1);
                const R gdh2 = dh > R(0) ? gl2 * inv_l1 : R(0);
                gl1 += -gl2 * l2 * inv_l1;
                gh00 += gdh2 * h11;
                gh11 += gdh2 * h00;
                gh01 += -R(2) * gdh2 * h01;
                const R inv_rad = rad > R(0) ? O::rcp(rad) : R(0);
                const R ghalf = gl1 * half * inv_rad;
                gh01 += gl1 * h01 * inv_rad;
                gh00 += R(0.5) * gl1 + R(0.5) * ghalf;
                gh11 += R(0.5) * gl1 - R(0.5) * ghalf;
            }
            const R gt2 = gh00 * f.A00 + gh01 * f.A01 + gh11 * f.A11;
            const R gA00 = gh00 * f.t2, gA01 = gh01 * f.t2, gA11 = gh11 * f.t2;
            gts += gt2 * (R(2) / R(3)) * f.ts;
            gcx += gA00 * (R(2) * f.cx - R(2) * px.d_dx) + gA01 * (f.cy - px.d_dy);
            gcy += gA11 * (R(2) * f.cy - R(2) * px.d_dy) + gA01 * (f.cx - px.d_dx);
        }
        // G, b from e_x, e_y, q
        R gex[3], gey[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            gex[k] = R(2) * gG00 * f.ex[k] + gG01 * f.ey[k] + gb0 * f.q[k];
            gey[k] = R(2) * gG11 * f.ey[k] + gG01 * f.ex[k] + gb1 * f.q[k];
            gq[k] += gb0 * f.ex[k] + gb1 * f.ey[k];
        }
        // e_i = ts (g_i - c_i du)
        const R ts = f.ts;
        R gxe = R(0), gye = R(0);
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            gts += gex[k] * (f.gx[k] - f.cx * f.du[k]) + gey[k] * (f.gy[k] - f.cy * f.du[k]);
            ggx[k] += ts * gex[k];
            ggy[k] += ts * gey[k];
            gxe += gex[k] * f.du[k];
            gye += gey[k] * f.du[k];
            gdu[k] += -ts * (f.cx * gex[k] + f.cy * gey[k]);
        }
        gcx += -ts * gxe;
        gcy += -ts * gye;
        // c_i = (du . g_i) inv_n
        R dgx = R(0), dgy = R(0);
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            gdu[k] += (gcx * f.gx[k] + gcy * f.gy[k]) * f.inv_n;
            ggx[k] += gcx * f.inv_n * f.du[k];
            ggy[k] += gcy * f.inv_n * f.du[k];
            dgx += f.du[k] * f.gx[k];
            dgy += f.du[k] * f.gy[k];
        }
        ginv_n += gcx * dgx + gcy * dgy;
    }
    // qq = q.q ; q = o_u + ts du
    const R *ou = gr.ou;
#pragma unroll
    for (int k = 0; k < 3; ++k) gq[k] += R(2) * gqq * f.q[k];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        gou_r[k] += gq[k];
        gts += gq[k] * f.du[k];
        gdu[k] += f.ts * gq[k];
    }
    // ts = -p inv_n ; p = o_u . du ; inv_n = 1/n ; n = du . du
    const R gp = -gts * f.inv_n;
    ginv_n += -gts * f.p;
    const R gn = -ginv_n * f.inv_n * f.inv_n;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        gou_r[k] += gp * f.du[k];
        gdu[k] += gp * ou[k] + R(2) * gn * f.du[k];
    }
    // du = W d, g_x = W dx, g_y = W dy
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        gou[a] += (float)gou_r[a];
#pragma unroll
        for (int b = 0; b < 3; ++b)
            gW[3 * a + b] += (float)(gdu[a] * R(px.d[b]) + (FILTER ? ggx[a] * R(px.dx[b]) + ggy[a] * R(px.dy[b]) : R(0)));
    }
    return (float)gsig;
}

}  // namespace conegs
