// Per pixel-Gaussian pair response (Sec. 4.1-4.2) in registers.
//
// One implementation, generic over the arithmetic type V, with a fixed
// sequence of correctly rounded operations (so the forward and the adjoint,
// which recomputes the forward's pairs, take the same compositing decisions):
//   float   every pair of an ordinary Gaussian;
//   double  near-degenerate flat Gaussians (effective scale ratio above
//           FLAT_RATIO): their whitening W has a row of length 1/s_min, so the
//           whitened camera centre o_u is large and t* and q = o_u + t* d_u
//           cancel.  Measured against the FP64 oracle, the FP32 form below
//           stays within ~2e-5 up to s_max/s_min = 250 at any viewing angle and
//           size, reaches ~9e-5 at 400 and ~3e-4 at 600 (small disks seen
//           face-on), hence the threshold of 200.
// FP32 uses the SFU approximations of reciprocal, reciprocal square root and
// 2^x (about 1-2 ulp, subnormals flushed), far inside the 1e-4 output tolerance;
// FP64 the correctly rounded operations.
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
// A = I + E K E^T; with an orthonormal basis [e1 e2] of span(E), E = [e1 e2] R:
//   det A = det(I + N),  q^T A^-1 q = |q_perp|^2 + q_E^T (I + N)^-1 q_E,
//   N = R K R^T, q_E = [e1 e2]^T q, q_perp = q - [e1 e2] q_E,
//   T = sigma_eff det(A)^-1/2 exp(-q^T A^-1 q / 2)                   (Eq. 9)
// No 3x3 matrix is formed.
#pragma once
#include "common.cuh"

namespace conegs {

// A Gaussian is "flat" (evaluated in FP64) when s_eff,max / s_eff,min > FLAT_RATIO
// (the effective scales of Eq. 10, after the floor).
constexpr float FLAT_RATIO = 200.0f;

// ---------------------------------------------------------------- arithmetic per type

// The special-function unit's approximations (reciprocal, reciprocal square
// root, 2^x) with subnormal inputs and results flushed to zero: one SFU
// instruction each, where the non-flushing forms add range scaling around it.
// Nothing the pair response decides rests on values that small: a response
// below 2^-126 lies far under the 1/255 opacity threshold, and the ray
// quantities that are inverted are bounded away from zero.
__device__ __forceinline__ float sfu_rcp(float a) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(a));
    return r;
}
__device__ __forceinline__ float sfu_rsqrt(float a) {
    float r;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(a));
    return r;
}
__device__ __forceinline__ float sfu_exp2(float a) {
    float r;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(a));
    return r;
}
// e^a = 2^(a log2 e)
__device__ __forceinline__ float sfu_exp(float a) { return sfu_exp2(__fmul_rn(a, 1.4426950408889634f)); }
// Smallest argument the guarded forms pass to the SFU: a zero argument gives
// a zero result (r2 * rsqrt(max(r2, tiny)) = 0) without a compare and select.
constexpr float SFU_TINY = 1e-36f;

template <typename V>
struct Ops;

template <>
struct Ops<float> {
    using B = bool;
    static __device__ __forceinline__ float S(float a) { return a; }
    static __device__ __forceinline__ B SB(bool a) { return a; }
    static __device__ __forceinline__ float add(float a, float b) { return __fadd_rn(a, b); }
    static __device__ __forceinline__ float sub(float a, float b) { return __fsub_rn(a, b); }
    static __device__ __forceinline__ float mul(float a, float b) { return __fmul_rn(a, b); }
    static __device__ __forceinline__ float fma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
    static __device__ __forceinline__ float neg(float a) { return -a; }
    static __device__ __forceinline__ float rcp(float a) { return sfu_rcp(a); }
    static __device__ __forceinline__ float rsqrt(float a) { return sfu_rsqrt(a); }
    // 1/sqrt(a) for a > 0; a = 0 (a zero vector's squared length) gives a finite
    // factor that keeps the vector's zero components zero
    static __device__ __forceinline__ float rsqrt0(float a) { return sfu_rsqrt(fmaxf(a, SFU_TINY)); }
    static __device__ __forceinline__ float sqrt(float a) { return sqrtf(a); }
    static __device__ __forceinline__ float exp(float a) { return sfu_exp(a); }
    static __device__ __forceinline__ float max(float a, float b) { return fmaxf(a, b); }
    static __device__ __forceinline__ B gt(float a, float b) { return a > b; }
    static __device__ __forceinline__ B eq(float a, float b) { return a == b; }
    static __device__ __forceinline__ B bor(B a, B b) { return a || b; }
    static __device__ __forceinline__ B bnot(B a) { return !a; }
    static __device__ __forceinline__ float sel(B c, float a, float b) { return c ? a : b; }
    // sqrt(r2) as r2 * rsqrt(r2) (0 at 0)
    static __device__ __forceinline__ float root(float r2) { return __fmul_rn(r2, sfu_rsqrt(fmaxf(r2, SFU_TINY))); }
};

template <>
struct Ops<double> {
    using B = bool;
    static __device__ __forceinline__ double S(double a) { return a; }
    static __device__ __forceinline__ B SB(bool a) { return a; }
    static __device__ __forceinline__ double add(double a, double b) { return __dadd_rn(a, b); }
    static __device__ __forceinline__ double sub(double a, double b) { return __dsub_rn(a, b); }
    static __device__ __forceinline__ double mul(double a, double b) { return __dmul_rn(a, b); }
    static __device__ __forceinline__ double fma(double a, double b, double c) { return __fma_rn(a, b, c); }
    static __device__ __forceinline__ double neg(double a) { return -a; }
    static __device__ __forceinline__ double rcp(double a) { return 1.0 / a; }
    static __device__ __forceinline__ double rsqrt(double a) { return ::rsqrt(a); }
    static __device__ __forceinline__ double rsqrt0(double a) { return a > 0.0 ? ::rsqrt(a) : 0.0; }
    static __device__ __forceinline__ double sqrt(double a) { return ::sqrt(a); }
    static __device__ __forceinline__ double exp(double a) { return ::exp(a); }
    static __device__ __forceinline__ double max(double a, double b) { return fmax(a, b); }
    static __device__ __forceinline__ B gt(double a, double b) { return a > b; }
    static __device__ __forceinline__ B eq(double a, double b) { return a == b; }
    static __device__ __forceinline__ B bor(B a, B b) { return a || b; }
    static __device__ __forceinline__ B bnot(B a) { return !a; }
    static __device__ __forceinline__ double sel(B c, double a, double b) { return c ? a : b; }
    static __device__ __forceinline__ double root(double r2) { return r2 > 0.0 ? ::sqrt(r2) : 0.0; }
};

// a . b of 3-vectors, in a fixed order of correctly rounded operations
template <typename V>
__device__ __forceinline__ V dot3v(V a0, V a1, V a2, V b0, V b1, V b2) {
    using O = Ops<V>;
    return O::fma(a2, b2, O::fma(a1, b1, O::mul(a0, b0)));
}

__device__ __forceinline__ float dot3(const float a[3], const float b[3]) {
    return dot3v(a[0], a[1], a[2], b[0], b[1], b[2]);
}

// ---------------------------------------------------------------- inputs

// The pixel's centre ray d and half-edge differentials, with the Gram terms of Eq. 12.
template <typename V>
struct PixelRaysT {
    V d[3], dx[3], dy[3];
    V d_dx, d_dy, dxdx, dxdy, dydy;
    float pc[2];          // pixel centre (i + 1/2, j + 1/2), for the pinhole pre-test
};
using PixelRays = PixelRaysT<float>;

__device__ __forceinline__ PixelRaysT<double> widen(const PixelRays &a) {
    PixelRaysT<double> p;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        p.d[k] = a.d[k];
        p.dx[k] = a.dx[k];
        p.dy[k] = a.dy[k];
    }
    // the Gram terms again in FP64
    p.d_dx = dot3v(p.d[0], p.d[1], p.d[2], p.dx[0], p.dx[1], p.dx[2]);
    p.d_dy = dot3v(p.d[0], p.d[1], p.d[2], p.dy[0], p.dy[1], p.dy[2]);
    p.dxdx = dot3v(p.dx[0], p.dx[1], p.dx[2], p.dx[0], p.dx[1], p.dx[2]);
    p.dxdy = dot3v(p.dx[0], p.dx[1], p.dx[2], p.dy[0], p.dy[1], p.dy[2]);
    p.dydy = dot3v(p.dy[0], p.dy[1], p.dy[2], p.dy[0], p.dy[1], p.dy[2]);
    p.pc[0] = a.pc[0];
    p.pc[1] = a.pc[1];
    return p;
}

// Everything of a Gaussian's view record the response needs: W_eff rows, o_u,
// sigma_eff, rho^2.
template <typename V>
struct GaussRec {
    V W[9], ou[3], sig, rho2;
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

// ---------------------------------------------------------------- Eq. 12: K = f(H')

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

// Both eigenvalues of H' above rho^2: K = (I - rho^2 H'^-1)/3.
template <typename V>
__device__ __forceinline__ void K_both(V h00, V h01, V h11, V dh, V rho2, V &k00, V &k01, V &k11) {
    using O = Ops<V>;
    const V third = O::S(1.0f / 3.0f);
    const V s = O::mul(rho2, O::rcp(dh));
    k00 = O::mul(O::fma(O::neg(s), h11, O::S(1.0f)), third);
    k11 = O::mul(O::fma(O::neg(s), h00, O::S(1.0f)), third);
    k01 = O::mul(O::mul(s, h01), third);
}

// Only the larger above rho^2: K = f(l1) (H' - l2 I)/(l1 - l2), f(l) = (l - rho^2)/(3 l).
template <typename V>
__device__ __forceinline__ void K_major(V h00, V h01, V h11, V l1, V l2, V rho2, V &k00, V &k01, V &k11) {
    using O = Ops<V>;
    const V sc = O::mul(O::sub(l1, rho2), O::rcp(O::mul(O::mul(O::S(3.0f), l1), O::sub(l1, l2))));
    k00 = O::mul(sc, O::sub(h00, l2));
    k11 = O::mul(sc, O::sub(h11, l2));
    k01 = O::mul(sc, h01);
}

// ---------------------------------------------------------------- the response

// Response of the pair in type V.  hit: false where t* <= T_NEAR (the pair is
// skipped; the call returns early).  With STORE the intermediates are copied to
// *st; the arithmetic is the same either way.
template <bool FILTER, bool STORE = false, typename V = float>
__device__ __forceinline__ void pair_eval(const GaussRec<V> &g, const bool additive, const PixelRaysT<V> &px, V &T,
                                          typename Ops<V>::B &hit, PairFwdT<V> *st = nullptr) {
    using O = Ops<V>;
    using B = typename O::B;
    const V *W = g.W;
    const V du0 = dot3v(W[0], W[1], W[2], px.d[0], px.d[1], px.d[2]);
    const V du1 = dot3v(W[3], W[4], W[5], px.d[0], px.d[1], px.d[2]);
    const V du2 = dot3v(W[6], W[7], W[8], px.d[0], px.d[1], px.d[2]);
    const V n = dot3v(du0, du1, du2, du0, du1, du2);
    const V inv_n = O::rcp(n);
    const V p = dot3v(g.ou[0], g.ou[1], g.ou[2], du0, du1, du2);
    const V ts = O::neg(O::mul(p, inv_n));
    hit = O::gt(ts, O::S(T_NEAR));
    if (!hit) return;
    const V q0 = O::fma(ts, du0, g.ou[0]), q1 = O::fma(ts, du1, g.ou[1]), q2 = O::fma(ts, du2, g.ou[2]);
    const V qq = dot3v(q0, q1, q2, q0, q1, q2);
    if constexpr (STORE) {
        st->du[0] = du0; st->du[1] = du1; st->du[2] = du2;
        st->inv_n = inv_n; st->p = p; st->ts = ts;
        st->q[0] = q0; st->q[1] = q1; st->q[2] = q2; st->qq = qq;
    }
    if constexpr (!FILTER) {
        T = O::mul(g.sig, O::exp(O::mul(O::S(-0.5f), qq)));
        if constexpr (STORE) st->T = T;
        return;
    } else {
        const V gx0 = dot3v(W[0], W[1], W[2], px.dx[0], px.dx[1], px.dx[2]);
        const V gx1 = dot3v(W[3], W[4], W[5], px.dx[0], px.dx[1], px.dx[2]);
        const V gx2 = dot3v(W[6], W[7], W[8], px.dx[0], px.dx[1], px.dx[2]);
        const V gy0 = dot3v(W[0], W[1], W[2], px.dy[0], px.dy[1], px.dy[2]);
        const V gy1 = dot3v(W[3], W[4], W[5], px.dy[0], px.dy[1], px.dy[2]);
        const V gy2 = dot3v(W[6], W[7], W[8], px.dy[0], px.dy[1], px.dy[2]);
        const V cx = O::mul(dot3v(du0, du1, du2, gx0, gx1, gx2), inv_n);
        const V cy = O::mul(dot3v(du0, du1, du2, gy0, gy1, gy2), inv_n);
        const V ncx = O::neg(cx), ncy = O::neg(cy);
        const V ex0 = O::mul(ts, O::fma(ncx, du0, gx0)), ex1 = O::mul(ts, O::fma(ncx, du1, gx1)),
                ex2 = O::mul(ts, O::fma(ncx, du2, gx2));
        const V ey0 = O::mul(ts, O::fma(ncy, du0, gy0)), ey1 = O::mul(ts, O::fma(ncy, du1, gy1)),
                ey2 = O::mul(ts, O::fma(ncy, du2, gy2));
        // Eq. 12: H' = t*^2/3 [f_i . f_j], f_i = delta_i - c_i d, and the case of K
        const V third = O::S(1.0f / 3.0f);
        const V t2 = O::mul(O::mul(ts, ts), third);
        const V A00 = O::fma(cx, O::sub(cx, O::mul(O::S(2.0f), px.d_dx)), px.dxdx);
        const V A01 = O::sub(O::fma(cx, O::sub(cy, px.d_dy), px.dxdy), O::mul(cy, px.d_dx));
        const V A11 = O::fma(cy, O::sub(cy, O::mul(O::S(2.0f), px.d_dy)), px.dydy);
        const V h00 = O::mul(t2, A00), h01 = O::mul(t2, A01), h11 = O::mul(t2, A11);
        const V mean = O::mul(O::S(0.5f), O::add(h00, h11));
        const V half = O::mul(O::S(0.5f), O::sub(h00, h11));
        const V l1 = O::add(mean, O::root(O::fma(half, half, O::mul(h01, h01))));
        const V dh = O::fma(h00, h11, O::neg(O::mul(h01, h01)));
        const V l2 = O::mul(O::max(dh, O::S(0.0f)), O::rcp(l1));   // smaller eigenvalue without cancellation
        const B id = O::bor(O::eq(g.rho2, O::S(0.0f)), O::SB(additive));
        const B none = O::bnot(O::gt(l1, g.rho2));
        const B both = O::gt(l2, g.rho2);
        // K for every case, chosen without a branch (the warp's lanes evaluate
        // different pairs, whose cases differ)
        V a00, a01, a11, c00, c01, c11;
        K_both(h00, h01, h11, dh, g.rho2, a00, a01, a11);
        K_major(h00, h01, h11, l1, l2, g.rho2, c00, c01, c11);
        V k00 = O::sel(both, a00, c00), k01 = O::sel(both, a01, c01), k11 = O::sel(both, a11, c11);
        k00 = O::sel(none, O::S(0.0f), k00);
        k01 = O::sel(none, O::S(0.0f), k01);
        k11 = O::sel(none, O::S(0.0f), k11);
        k00 = O::sel(id, third, k00);
        k01 = O::sel(id, O::S(0.0f), k01);
        k11 = O::sel(id, third, k11);
        const int kc = id ? 0 : none ? 3 : both ? 1 : 2;
        // Eq. 9 in an orthonormal basis (e1, e2) of span(E): E = [e1 e2] R with
        // R = [[r00, r01], [0, r11]] (Gram-Schmidt), N = R K R^T, so that
        //   det A = det(I + N),  q^T A^-1 q = |q_perp|^2 + q_E^T (I + N)^-1 q_E,
        // q_E = (e1.q, e2.q), q_perp = q - e1 (e1.q) - e2 (e2.q).  No difference of
        // two large quadratic forms is taken: q_perp is formed as a vector, so its
        // rounding stays at the size of q's components, which keeps FP32 accurate
        // for strongly anisotropic Gaussians at grazing angles.
        const V r00s = dot3v(ex0, ex1, ex2, ex0, ex1, ex2);
        const V i0 = O::rsqrt0(r00s);
        const V e10 = O::mul(ex0, i0), e11 = O::mul(ex1, i0), e12 = O::mul(ex2, i0);
        const V r00 = O::mul(r00s, i0);
        const V r01 = dot3v(ey0, ey1, ey2, e10, e11, e12);
        const V nr01 = O::neg(r01);
        const V w0 = O::fma(nr01, e10, ey0), w1 = O::fma(nr01, e11, ey1), w2 = O::fma(nr01, e12, ey2);
        const V r11s = dot3v(w0, w1, w2, w0, w1, w2);
        const V i1 = O::rsqrt0(r11s);
        const V e20 = O::mul(w0, i1), e21 = O::mul(w1, i1), e22 = O::mul(w2, i1);
        const V r11 = O::mul(r11s, i1);
        const V qe1 = dot3v(q0, q1, q2, e10, e11, e12), qe2 = dot3v(q0, q1, q2, e20, e21, e22);
        const V nq1 = O::neg(qe1), nq2 = O::neg(qe2);
        const V qp0 = O::fma(nq2, e20, O::fma(nq1, e10, q0)), qp1 = O::fma(nq2, e21, O::fma(nq1, e11, q1)),
                qp2 = O::fma(nq2, e22, O::fma(nq1, e12, q2));
        const V qperp = dot3v(qp0, qp1, qp2, qp0, qp1, qp2);
        const V RK00 = O::fma(r00, k00, O::mul(r01, k01)), RK01 = O::fma(r00, k01, O::mul(r01, k11));
        const V N11 = O::fma(RK00, r00, O::mul(RK01, r01));
        const V N12 = O::mul(RK01, r11);
        const V N22 = O::mul(O::mul(r11, k11), r11);
        const V a1 = O::add(O::S(1.0f), N11), a2 = O::add(O::S(1.0f), N22);
        const V detA = O::fma(a1, a2, O::neg(O::mul(N12, N12)));
        const V num = O::fma(O::mul(qe1, qe1), a2,
                             O::fma(O::mul(qe2, qe2), a1, O::mul(O::mul(O::S(-2.0f), O::mul(qe1, qe2)), N12)));
        const V rdet = O::rsqrt(detA);
        const V Q = O::max(O::fma(num, O::mul(rdet, rdet), qperp), O::S(0.0f));
        T = O::mul(O::mul(g.sig, rdet), O::exp(O::mul(O::S(-0.5f), Q)));
        if constexpr (STORE) {
            // what the adjoint differentiates: the same T through G = E^T E, b = E^T q,
            // M = I + G K, P = K adj(M): q^T A^-1 q = max(|q|^2 - b^T P b / det M, |q|^2 / det M)
            const V G00 = dot3v(ex0, ex1, ex2, ex0, ex1, ex2);
            const V G01 = dot3v(ex0, ex1, ex2, ey0, ey1, ey2);
            const V G11 = dot3v(ey0, ey1, ey2, ey0, ey1, ey2);
            const V b0 = dot3v(ex0, ex1, ex2, q0, q1, q2);
            const V b1 = dot3v(ey0, ey1, ey2, q0, q1, q2);
            const V m00 = O::fma(G00, k00, O::fma(G01, k01, O::S(1.0f))), m01 = O::fma(G00, k01, O::mul(G01, k11));
            const V m10 = O::fma(G01, k00, O::mul(G11, k01)), m11 = O::fma(G01, k01, O::fma(G11, k11, O::S(1.0f)));
            const V det = O::fma(m00, m11, O::neg(O::mul(m01, m10)));
            const V p00 = O::fma(k00, m11, O::neg(O::mul(k01, m10))), p01 = O::fma(k01, m00, O::neg(O::mul(k00, m01)));
            const V p10 = O::fma(k01, m11, O::neg(O::mul(k11, m10))), p11 = O::fma(k11, m00, O::neg(O::mul(k01, m01)));
            const V bPb =
                O::fma(O::mul(b0, b0), p00, O::fma(O::mul(b0, b1), O::add(p01, p10), O::mul(O::mul(b1, b1), p11)));
            const V inv_det = O::rcp(det);
            const V Qa = O::fma(O::neg(bPb), inv_det, qq), Qb = O::mul(qq, inv_det);
            st->m00 = m00; st->m01 = m01; st->m10 = m10; st->m11 = m11;
            st->p00 = p00; st->p01 = p01; st->p10 = p10; st->p11 = p11;
            st->det = det; st->bPb = bPb; st->inv_det = inv_det;
            st->clamped = !(Qa >= Qb);
            st->gx[0] = gx0; st->gx[1] = gx1; st->gx[2] = gx2;
            st->gy[0] = gy0; st->gy[1] = gy1; st->gy[2] = gy2;
            st->cx = cx; st->cy = cy;
            st->ex[0] = ex0; st->ex[1] = ex1; st->ex[2] = ex2;
            st->ey[0] = ey0; st->ey[1] = ey1; st->ey[2] = ey2;
            st->G00 = G00; st->G01 = G01; st->G11 = G11; st->b0 = b0; st->b1 = b1;
            st->kcase = kc;
            st->k00 = k00; st->k01 = k01; st->k11 = k11;
            st->t2 = t2; st->A00 = A00; st->A01 = A01; st->A11 = A11;
            st->h00 = h00; st->h01 = h01; st->h11 = h11;
            st->T = T;
        }
    }
}

// Scalar convenience form: true when the pair is evaluated (t* > T_NEAR), T the response.
template <bool FILTER, bool STORE = false, typename R = float>
__device__ __forceinline__ bool pair_response(const GaussRec<R> &g, const bool additive, const PixelRaysT<R> &px,
                                              float &Tout, PairFwdT<R> *st = nullptr) {
    R T = R(0);
    bool hit;
    pair_eval<FILTER, STORE, R>(g, additive, px, T, hit, st);
    Tout = (float)T;
    return hit;
}

// ---------------------------------------------------------------- the rasteriser's pre-test

// Visual-cone pre-test (view record words u, g, C; see preprocess.cu): a pixel
// ray d with -1 + g.e + e^T C e > 1e-3, e = d - u, cannot reach alpha >= 1/255
// with the Gaussian.  Returns true when the pair must be evaluated.  The same
// operations in the forward and the adjoint.
template <typename V>
__device__ __forceinline__ typename Ops<V>::B pretest(V u0, V u1, V u2, V g0, V g1, V g2, V C00, V C11, V C22, V C01,
                                                      V C02, V C12, const V d[3]) {
    using O = Ops<V>;
    const V e0 = O::sub(d[0], u0), e1 = O::sub(d[1], u1), e2 = O::sub(d[2], u2);
    const V qa = O::fma(C02, e2, O::fma(C01, e1, O::mul(C00, e0)));
    const V qb = O::fma(C12, e2, O::mul(C11, e1));
    const V quad = O::fma(O::mul(C22, e2), e2, O::fma(qb, e1, O::mul(qa, e0)));
    const V lin = O::fma(g2, e2, O::fma(g1, e1, O::fma(g0, e0, O::S(-1.0f))));
    return O::bnot(O::gt(O::add(lin, quad), O::S(1e-3f)));
}

// Pinhole form of the same pre-test (view record words r4 = (c_x, c_y, G00, 2 G01),
// r5.xy = (G11, t); see preprocess.cu): the pixel centre p must satisfy
// (p - c)^T G (p - c) <= t, the ellipse the visual cone cuts from the image
// plane, in pixels.  Fixed, correctly rounded operations (the forward and the
// adjoint take the same decision).
__device__ __forceinline__ bool pretest_pix(const float4 r4, const float2 r5, const float pc[2]) {
    const float ex = __fsub_rn(pc[0], r4.x), ey = __fsub_rn(pc[1], r4.y);
    const float t = __fmaf_rn(r4.w, ey, __fmul_rn(r4.z, ex));            // G00 ex + 2 G01 ey
    const float q = __fmaf_rn(t, ex, __fmul_rn(__fmul_rn(r5.x, ey), ey));
    return q <= r5.y;
}

// The pre-test of staged record b (records staged as s[word][entry]) against a
// pixel: PIX selects the pinhole form.
template <bool PIX, int N>
__device__ __forceinline__ bool staged_pretest(const float4 (*s)[N], int b, const PixelRays &px) {
    if constexpr (PIX) {
        const float4 r4 = s[4][b];
        const float2 r5 = *reinterpret_cast<const float2 *>(&s[5][b]);
        return pretest_pix(r4, r5, px.pc);
    } else {
        const float4 r4 = s[4][b], r5 = s[5][b], r6 = s[6][b];
        return pretest<float>(r4.x, r4.y, r4.z, r4.w, r5.x, r5.y, r5.z, r5.w, r6.x, r6.y, r6.z, r6.w, px.d);
    }
}

}  // namespace conegs
