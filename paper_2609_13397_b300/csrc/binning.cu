// K3: conservative angular-tile binning.
//
// The paper has no binning stage; this one is the library's own rule,
// written so that its decisions are reproducible bit for bit: every
// operation below is one correctly rounded FP32 operation (_rn intrinsics,
// no contraction) in a fixed order, and the transcendental functions the
// rule needs are replaced by fixed polynomials (Taylor series of exp, sin
// and cos).  The rule:
//   * tile cone: axis a_t = ray of the tile centre; half-angle gamma from the
//     largest chord |a_t - d_p| over the tile's valid pixel rays, inflated;
//     m_t >= (|delta_x|^2 + |delta_y|^2)/3 over the tile;
//   * Gaussian bound: alpha >= 1/255 needs q^T A^-1 q <= kappa^2 =
//     2 ln(255 sigma), so the world distance from mu to a contributing
//     centre ray is at most kappa sqrt(s_max^2 + t*^2 m) (A >= I and
//     Sigma_render <= Sigma_fp,eff, Eq. 9 and 12), with
//     t* <= (L + kappa s_max) / (1 - kappa (1 + s_max/s_min) sqrt(m)) and
//     |x* - mu| <= 255 kappa s_max (from det A <= (255 sigma)^2);
//   * cone test: the angle between mu - o and a_t is at most beta + gamma,
//     sin(beta) = bound / L (chord form);
//   * silhouette test (rule.cuh): the Gaussian's bounding ellipsoid seen from
//     the camera centre is an elliptic cone; its trace (an ellipse on a
//     pinhole's image plane, or in the gnomonic plane around mu - o for a
//     fisheye) must reach the tile's pixel-centre rectangle (pinhole) or the
//     disc bounding the tile's rays (fisheye).
// A pair is kept when both tests pass.  Candidates come from boxes (the
// cone's image, cut to the ellipse's box on pinholes) or, without a box, from
// super-tiles of 8x8 tiles pruned by a cheap conservative cone test (fast
// math, wide margins); the exact tests decide for every candidate.
#include "rule.cuh"

namespace conegs {

// ---------------------------------------------------------------- tile tables

// One CTA of TILE*TILE threads per tile; thread = pixel.  Max-reductions are
// exact and order independent.
__global__ void __launch_bounds__(TILE_PX) tile_table_kernel(CamParams c, float *__restrict__ table) {
    const int t = blockIdx.x;
    const int tx = t % c.tiles_x, ty = t / c.tiles_x;
    const int i = tx * TILE + (threadIdx.x % TILE), j = ty * TILE + (threadIdx.x / TILE);
    __shared__ float s_a[3];
    if (threadIdx.x == 0) {
        float a[3];
        rule_dir(c, (float)(TILE * tx + TILE / 2), (float)(TILE * ty + TILE / 2), a);
        s_a[0] = a[0]; s_a[1] = a[1]; s_a[2] = a[2];
    }
    __syncthreads();
    float ch2 = -1.0f, mm = 0.0f;
    if (i < c.W && j < c.H) {
        float x = (float)i + 0.5f, y = (float)j + 0.5f;
        if (rule_valid(c, x, y)) {
            float d[3], ex[3], ey[3];
            rule_dir(c, x, y, d);
            float e0 = r_sub(s_a[0], d[0]), e1 = r_sub(s_a[1], d[1]), e2 = r_sub(s_a[2], d[2]);
            ch2 = r_add(r_add(r_mul(e0, e0), r_mul(e1, e1)), r_mul(e2, e2));
            rule_edge(c, x, y, d, 0, ex);
            rule_edge(c, x, y, d, 1, ey);
            mm = r_div(r_add(r_add(r_add(r_mul(ex[0], ex[0]), r_mul(ex[1], ex[1])), r_mul(ex[2], ex[2])),
                       r_add(r_add(r_mul(ey[0], ey[0]), r_mul(ey[1], ey[1])), r_mul(ey[2], ey[2]))),
                    3.0f);
        }
    }
    for (int off = 16; off > 0; off >>= 1) {
        ch2 = fmaxf(ch2, __shfl_xor_sync(0xffffffffu, ch2, off));
        mm = fmaxf(mm, __shfl_xor_sync(0xffffffffu, mm, off));
    }
    constexpr int NW = (TILE_PX + 31) / 32;
    __shared__ float s_ch[NW], s_mm[NW];
    if ((threadIdx.x & 31) == 0) {
        s_ch[threadIdx.x >> 5] = ch2;
        s_mm[threadIdx.x >> 5] = mm;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        float chm = s_ch[0], mmm = s_mm[0];
        for (int w = 1; w < NW; ++w) {
            chm = fmaxf(chm, s_ch[w]);
            mmm = fmaxf(mmm, s_mm[w]);
        }
        float *o = table + 6 * (size_t)t;
        o[0] = s_a[0]; o[1] = s_a[1]; o[2] = s_a[2];
        if (chm < 0.0f) {
            o[3] = -1.0f; o[4] = 0.0f; o[5] = 0.0f;
        } else {
            float sg = r_add(r_mul(r_sqrt(chm), 0.5f), 2e-6f);
            sg = fminf(sg, 1.0f);
            o[3] = sg;
            o[4] = r_sqrt(r_sub(1.0f, r_mul(sg, sg)));
            o[5] = r_mul(mmm, 1.01f);
        }
    }
}

// Super-tile cones containing every child tile cone (pruning only; extra margins).
__global__ void super_table_kernel(CamParams c, const float *__restrict__ table, float *__restrict__ super) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= c.supers_x * c.supers_y) return;
    const int sx = s % c.supers_x, sy = s / c.supers_x;
    float a[3];
    rule_dir(c, (float)(TILE * SUPER * sx + TILE * SUPER / 2), (float)(TILE * SUPER * sy + TILE * SUPER / 2), a);
    float best = -1.0f, mmax = 0.0f;
    for (int cy = 0; cy < SUPER; ++cy)
        for (int cx = 0; cx < SUPER; ++cx) {
            int tx = sx * SUPER + cx, ty = sy * SUPER + cy;
            if (tx >= c.tiles_x || ty >= c.tiles_y) continue;
            const float *t = table + 6 * (size_t)(ty * c.tiles_x + tx);
            if (t[3] < 0.0f) continue;
            float e0 = a[0] - t[0], e1 = a[1] - t[1], e2 = a[2] - t[2];
            float sa = 0.5f * sqrtf(e0 * e0 + e1 * e1 + e2 * e2);
            sa = fminf(sa, 1.0f);
            float ca = sqrtf(fmaxf(1.0f - sa * sa, 0.0f));
            float shalf = sa * t[4] + ca * t[3];      // sin((alpha + gamma)/2)
            float chalf = ca * t[4] - sa * t[3];      // cos((alpha + gamma)/2)
            if (chalf < 1e-3f) shalf = 1.0f;
            best = fmaxf(best, shalf);
            mmax = fmaxf(mmax, t[5]);
        }
    float *o = super + 6 * (size_t)s;
    o[0] = a[0]; o[1] = a[1]; o[2] = a[2];
    if (best < 0.0f) {
        o[3] = -1.0f; o[4] = 0.0f; o[5] = 0.0f;
        return;
    }
    float sg = fminf(best * 1.0001f + 1e-6f, 1.0f);
    o[3] = sg;
    o[4] = sqrtf(fmaxf(1.0f - sg * sg, 0.0f));
    o[5] = mmax * 1.0001f;
}

// Camera-wide bounds over the tiles: out[0] = max m_t (footprint, for the
// rasteriser's per-pixel pre-test), out[1] = max sin(gamma_t / 2) (tile cone
// half-angle, for the binning candidate box).  Fisheye cameras also get
// out[2 + j], j = 0..16: the largest sin(gamma_t / 2) over the tiles whose axis
// lies within theta_lim j / 16 of the optical axis (a non-decreasing envelope;
// tile cones grow toward a fisheye's rim).  out[MCAM_MMIN]: the smallest m over
// the valid tiles (3e38 without one).  out[19]: the half-angle (rad,
// widened) of a cone around the optical axis that contains every tile cone.
constexpr int GAMMA_BANDS = 16;

__global__ void max_m_kernel(CamParams c, const float *__restrict__ table, int nt, float *__restrict__ out) {
    __shared__ unsigned int s_band[GAMMA_BANDS + 1];
    __shared__ unsigned int s_reach;
    if (threadIdx.x <= GAMMA_BANDS) s_band[threadIdx.x] = 0u;
    if (threadIdx.x == 0) s_reach = 0u;
    __syncthreads();
    float m = 0.0f, g = 0.0f, reach = 0.0f, mlo = 3.0e38f;
    for (int t = threadIdx.x; t < nt; t += blockDim.x) {
        const float *r = table + 6 * (size_t)t;
        m = fmaxf(m, r[5]);
        g = fmaxf(g, r[3]);
        if (r[3] >= 0.0f) {
            mlo = fminf(mlo, r[5]);
            // the camera's cone: every tile cone lies within `reach` of the optical axis
            const float cz = r[0] * c.R[2] + r[1] * c.R[5] + r[2] * c.R[8];
            reach = fmaxf(reach, acosf(fminf(fmaxf(cz, -1.0f), 1.0f)) + 2.0f * asinf(fminf(r[3], 1.0f)));
        }
        if (c.model != 0 && r[3] >= 0.0f) {
            const float cz = r[0] * c.R[2] + r[1] * c.R[5] + r[2] * c.R[8];
            const float th = acosf(fminf(fmaxf(cz, -1.0f), 1.0f));
            // the band index rounds up (with margin), so band j covers every axis within its bound
            const int j = min(GAMMA_BANDS, max(0, (int)ceilf(th / c.thlim * GAMMA_BANDS * 1.0001f + 1e-4f)));
            atomicMax(&s_band[j], __float_as_uint(r[3]));    // non-negative floats order as their bits
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
        g = fmaxf(g, __shfl_xor_sync(0xffffffffu, g, o));
        reach = fmaxf(reach, __shfl_xor_sync(0xffffffffu, reach, o));
        mlo = fminf(mlo, __shfl_xor_sync(0xffffffffu, mlo, o));
    }
    if ((threadIdx.x & 31) == 0) atomicMax(&s_reach, __float_as_uint(reach));   // non-negative: bit order
    __shared__ float sm[32], sg[32], slo[32];
    if ((threadIdx.x & 31) == 0) {
        sm[threadIdx.x >> 5] = m;
        sg[threadIdx.x >> 5] = g;
        slo[threadIdx.x >> 5] = mlo;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) {
            m = fmaxf(m, sm[w]);
            g = fmaxf(g, sg[w]);
            mlo = fminf(mlo, slo[w]);
        }
        m = fmaxf(m, sm[0]);
        g = fmaxf(g, sg[0]);
        mlo = fminf(mlo, slo[0]);
        out[0] = m;
        out[1] = g;
        out[MCAM_MMIN] = mlo;     // 3e38 without a valid tile
        float env = 0.0f;
        for (int j = 0; j <= GAMMA_BANDS; ++j) {
            env = c.model != 0 ? fmaxf(env, __uint_as_float(s_band[j])) : g;
            out[2 + j] = env;
        }
        out[3 + GAMMA_BANDS] = __uint_as_float(s_reach) * 1.001f + 1e-4f;
    }
}

// ---------------------------------------------------------------- Gaussian bounds

__global__ void gauss_scene_rule_kernel(SceneParams sp, float *__restrict__ binrec) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= sp.n) return;
    float ls[3] = {sp.log_scales[3 * i], sp.log_scales[3 * i + 1], sp.log_scales[3 * i + 2]};
    float logit = load_scalar(sp.logits, i, sp.storage);
    float rho2 = sp.rho2 ? sp.rho2[i] : 0.0f;
    float rec[6];
    rule_gauss_scene(ls, logit, rho2, rec);
#pragma unroll
    for (int k = 0; k < 6; ++k) binrec[BINREC * i + k] = rec[k];
    const float q[4] = {sp.quats[4 * i], sp.quats[4 * i + 1], sp.quats[4 * i + 2], sp.quats[4 * i + 3]};
    float S[6];
    rule_gauss_sigma(q, ls, rho2, S);
#pragma unroll
    for (int k = 0; k < 6; ++k) binrec[BINREC * i + 6 + k] = S[k];
}

// Per view: u, L (float4) and the view flag (0 culled, 1 normal, 2 pass-all).
__global__ void gauss_view_rule_kernel(CamParams c, SceneParams sp, float4 *__restrict__ gview,
                                       uint8_t *__restrict__ gflag) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= sp.n) return;
    float mu[3] = {sp.means[3 * i], sp.means[3 * i + 1], sp.means[3 * i + 2]};
    float flag = sp.binrec[BINREC * i + 5], u[3], L;
    rule_gauss_view(c, mu, flag, u, L);
    gview[i] = make_float4(u[0], u[1], u[2], L);
    gflag[i] = (uint8_t)flag;
}

// ---------------------------------------------------------------- count / emit

// Cheap conservative prefilter (fast math, wide margins): the Gaussian's cone
// (half-angle beta from the camera's largest footprint, given as sin/cos of
// beta/2) against a tile or super-tile cone.  Everything the exact rule keeps
// passes here; only survivors are given to the exact rule.
__device__ __forceinline__ bool cone_prefilter(const float4 gv, const float2 half, const float *t) {
    if (t[3] < 0.0f) return false;
    const float e0 = gv.x - t[0], e1 = gv.y - t[1], e2 = gv.z - t[2];
    const float ch2 = e0 * e0 + e1 * e1 + e2 * e2;
    const float sphi = half.x * t[4] + half.y * t[3];     // sin((beta + gamma)/2)
    const float lim = 2.0f * sphi * 1.001f + 2e-5f;
    return ch2 <= lim * lim || half.y < 1e-3f;
}

// A tile's cone record with its footprint bound m raised to mzf (the z/f
// variant's bound; 0 otherwise, which leaves the record unchanged).
__device__ __forceinline__ void tile_record(const float *__restrict__ table, uint32_t tile, float mzf, float t[6]) {
#pragma unroll
    for (int k = 0; k < 6; ++k) t[k] = table[6 * (size_t)tile + k];
    t[5] = fmaxf(t[5], mzf);
}

// Tiles whose centre (TILE t + TILE/2 in pixel coordinates) lies within half a
// pixel of [xl, xh] x [yl, yh] (the margin is far above the FP32 error of the
// box bounds), clamped to the image.
__device__ __forceinline__ void tile_range(const CamParams &c, float xl, float xh, float yl, float yh, int &tx0,
                                           int &tx1, int &ty0, int &ty1) {
    const float lim = 1e8f;
    tx0 = max((int)ceilf(fmaxf((xl - 0.5f * TILE - 0.5f) / TILE, -lim)), 0);
    tx1 = min((int)floorf(fminf((xh - 0.5f * TILE + 0.5f) / TILE, lim)), c.tiles_x - 1);
    ty0 = max((int)ceilf(fmaxf((yl - 0.5f * TILE - 0.5f) / TILE, -lim)), 0);
    ty1 = min((int)floorf(fminf((yh - 0.5f * TILE + 0.5f) / TILE, lim)), c.tiles_y - 1);
}

// Pinhole cameras: the tiles whose centre ray lies within angle beta + gamma_max
// of the Gaussian's direction u (a superset of what cone_prefilter keeps, with
// margin) have their centre pixel inside the image of that cone on the plane
// z = 1 of the camera.  For a cone of half-angle theta around the unit camera-
// frame axis v (v_z > sin theta) that image is an ellipse; its dual conic is
// v v^T - sin^2(theta) I, whose tangent lines x = const give
//   x = (v_x v_z -+ s sqrt(v_x^2 + v_z^2 - s^2)) / (v_z^2 - s^2),  s = sin theta
// and the same in y.  Returns false (use the super-tile walk) when the cone
// reaches within about 1 degree of the image plane's horizon.
__device__ __forceinline__ bool pinhole_tile_box(const CamParams &c, const float4 gv, const float2 half,
                                                 const float sg_max, int &tx0, int &tx1, int &ty0, int &ty1) {
    // camera-frame axis: R^T u (R maps camera to world)
    const float v0 = c.R[0] * gv.x + c.R[3] * gv.y + c.R[6] * gv.z;
    const float v1 = c.R[1] * gv.x + c.R[4] * gv.y + c.R[7] * gv.z;
    const float v2 = c.R[2] * gv.x + c.R[5] * gv.y + c.R[8] * gv.z;
    // sin((beta + gamma_max)/2), widened beyond the prefilter's own margin
    const float cg = sqrtf(fmaxf(1.0f - sg_max * sg_max, 0.0f));
    const float sh = fminf((half.x * cg + half.y * sg_max) * 1.002f + 3e-5f, 1.0f);
    if (!(sh < 0.7f)) return false;                                // theta = 2 asin(sh) must stay below 90 degrees
    const float s = 2.0f * sh * sqrtf(fmaxf(1.0f - sh * sh, 0.0f));   // sin theta
    if (!(v2 > s + 0.02f)) return false;
    const float den = v2 * v2 - s * s;
    // FP32 error of the extremes grows like 1e-6 / den (normalised units); below
    // den = 0.05 (a cone near the horizon) the super-tile walk is used instead
    if (!(den >= 0.05f)) return false;
    const float rx = s * sqrtf(fmaxf(v0 * v0 + v2 * v2 - s * s, 0.0f));
    const float ry = s * sqrtf(fmaxf(v1 * v1 + v2 * v2 - s * s, 0.0f));
    const float inv = 1.0f / den;
    const float xl = c.fx * ((v0 * v2 - rx) * inv) + c.cx, xh = c.fx * ((v0 * v2 + rx) * inv) + c.cx;
    const float yl = c.fy * ((v1 * v2 - ry) * inv) + c.cy, yh = c.fy * ((v1 * v2 + ry) * inv) + c.cy;
    tile_range(c, xl, xh, yl, yh, tx0, tx1, ty0, ty1);
    return true;
}

// Kannala-Brandt cameras: a direction at polar angle theta (from the optical
// axis) and azimuth a images at normalised radius r(theta) = theta (1 + k1
// theta^2 + ... + k4 theta^8) (increasing on [0, theta_lim]) and azimuth a, so
// along any path on the unit sphere the image moves by at most max(r', r /
// sin theta) per unit of arc.  Every direction within Theta of the axis v is
// joined to v by an arc of length <= Theta that stays at polar angles <= phi +
// Theta (phi: the axis's), so its image lies within lip(phi + Theta) Theta of
// v's image.  A tile centre outside the valid circle has its axis clamped to
// theta_lim, so cones reaching theta_lim use the super-tile walk instead.
__device__ __forceinline__ float kb_radius(const CamParams &c, float th) {
    const float t2 = th * th;
    return th * (1.0f + t2 * (c.k[0] + t2 * (c.k[1] + t2 * (c.k[2] + t2 * c.k[3]))));
}

__device__ __forceinline__ bool kb_tile_box(const CamParams &c, const float4 gv, const float2 half,
                                            const float *__restrict__ mcam, int &tx0, int &tx1, int &ty0,
                                            int &ty1) {
    const float v0 = c.R[0] * gv.x + c.R[3] * gv.y + c.R[6] * gv.z;
    const float v1 = c.R[1] * gv.x + c.R[4] * gv.y + c.R[7] * gv.z;
    const float v2 = c.R[2] * gv.x + c.R[5] * gv.y + c.R[8] * gv.z;
    // the largest tile cone among the tiles this Gaussian can reach: tile axes lie
    // within phi + beta + gamma_max of the optical axis (gamma_max of the camera)
    float sg_max = mcam[1];
    {
        const float sphi0 = sqrtf(v0 * v0 + v1 * v1);
        const float reach = atan2f(sphi0, v2) + 2.0f * asinf(fminf(half.x, 1.0f)) + 2.0f * asinf(fminf(sg_max, 1.0f));
        const int j = (int)ceilf(reach / c.thlim * GAMMA_BANDS * 1.0001f + 1e-4f);
        if (j <= GAMMA_BANDS) sg_max = fminf(sg_max, mcam[2 + max(j, 0)]);
    }
    const float cg = sqrtf(fmaxf(1.0f - sg_max * sg_max, 0.0f));
    const float sh = fminf((half.x * cg + half.y * sg_max) * 1.002f + 3e-5f, 1.0f);
    if (!(sh < 0.7f)) return false;
    const float Th = 2.0f * asinf(sh) + 2e-3f;
    const float sphi = sqrtf(v0 * v0 + v1 * v1);
    const float phi = atan2f(sphi, v2);
    const float thi = phi + Th;
    if (!(thi < c.thlim - 1e-3f)) return false;
    const int j = min(16, (int)ceilf(thi / c.thlim * 16.0f + 1e-3f));
    const float rad = c.lip[j] * Th * 1.001f + 1e-5f;
    const float sc = sphi > 1e-6f ? kb_radius(c, phi) / sphi : 1.0f;   // r(phi) / sin(phi)
    const float xn = v0 * sc, yn = v1 * sc;
    tile_range(c, c.fx * (xn - rad) + c.cx, c.fx * (xn + rad) + c.cx, c.fy * (yn - rad) + c.cy,
               c.fy * (yn + rad) + c.cy, tx0, tx1, ty0, ty1);
    return true;
}

// ---------------------------------------------------------------- unscented-transform binning
//
// The alternative binning backbone of the 3DGUT family the paper renders with
// (Sec. 3): each Gaussian is bounded on the image by an unscented transform of
// its floored 3D distribution through the camera's own model, and a tile is
// kept when its pixel-centre rectangle meets the ellipse of alpha >= 1/255.
// The response (Eq. 9) is unchanged.  Definition (scaled UT with alpha = 1,
// beta = 2, kappa = 0, n = 3): sigma points mu and mu +- sqrt(3) s_eff,i R_i,
// mean weights 0 and 1/6, covariance weights 2 and 1/6; Sigma_2 gets I/12 px^2
// (the half-pixel footprint of Eq. 8 on the image); k^2 = 2 ln(255 sigma_eff).
// Gaussians with a sigma point outside the camera's domain (pinhole p_z <
// 0.1 |p|, fisheye polar angle > theta_lim) keep the angular-tile rule.
//
// The ellipse is formed in the count pass only and kept in the bin cache when
// the emit pass has to test tiles again, so both passes take every decision
// from the same floats; the tile test is a fixed sequence of correctly rounded
// operations, identical in both passes.
struct GaussArgs {
    const float4 *ell;      // [n][3] the angular-tile rule's silhouette ellipse (view records)
    const float *means;     // [n][3] (UT only)
    const float *W;         // [n][9] W_eff = S_eff^-1 R^T (UT only)
    const float *sig_eff;   // [n] (UT only)
};

constexpr float UT_COSMIN = 0.1f;
constexpr float UT_VLP = 1.0f / 12.0f;
constexpr uint32_t CACHE_UT = 2u;      // cache header .w: UT box and ellipse kept, tiles tested again

// Image of a camera-frame point under the fisheye model relative to the
// principal point (pixels); the caller has checked theta <= theta_lim.
__device__ __forceinline__ float2 ut_kb_image(const CamParams &c, float px, float py, float pz) {
    const float rho = sqrtf(px * px + py * py);
    const float th = atan2f(rho, pz);
    const float sc = rho > 0.0f ? kb_radius(c, th) / rho : 1.0f / pz;
    return make_float2(c.fx * (sc * px), c.fy * (sc * py));
}

// The UT image ellipse of Gaussian gid: e = (ybar_x, ybar_y, A, B, C) with
// [[A,B],[B,C]] = Sigma_2^-1, q = (k^2, -B/C, -B/A), and the candidate tile box.
// Returns false when a sigma point leaves the camera's domain.
__device__ bool ut_ellipse(const CamParams &c, const GaussArgs &ua, uint32_t gid, float e[5], float4 &q, int &tx0,
                           int &tx1, int &ty0, int &ty1) {
    const float m0 = ua.means[3 * (size_t)gid] - c.o[0], m1 = ua.means[3 * (size_t)gid + 1] - c.o[1],
                m2 = ua.means[3 * (size_t)gid + 2] - c.o[2];
    // camera frame (R maps camera to world): p = R^T (mu - o)
    const float p0x = c.R[0] * m0 + c.R[3] * m1 + c.R[6] * m2;
    const float p0y = c.R[1] * m0 + c.R[4] * m1 + c.R[7] * m2;
    const float p0z = c.R[2] * m0 + c.R[5] * m1 + c.R[8] * m2;
    float D[3][3];   // camera-frame sigma offsets sqrt(3) s_i R_i = sqrt(3) row_i(W) / |row_i(W)|^2
    const float *W = ua.W + 9 * (size_t)gid;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        const float w0 = W[3 * i], w1 = W[3 * i + 1], w2 = W[3 * i + 2];
        const float f = 1.7320508f / (w0 * w0 + w1 * w1 + w2 * w2);
        D[i][0] = f * (c.R[0] * w0 + c.R[3] * w1 + c.R[6] * w2);
        D[i][1] = f * (c.R[1] * w0 + c.R[4] * w1 + c.R[7] * w2);
        D[i][2] = f * (c.R[2] * w0 + c.R[5] * w1 + c.R[8] * w2);
    }
    // domain of all seven points
    const float kb_c2 = cosf(c.thlim);
    bool ok = true;
#pragma unroll
    for (int j = 0; j < 7; ++j) {
        const int i = (j - 1) >> 1;
        const float sg = (j & 1) ? 1.0f : -1.0f;
        const float px = j == 0 ? p0x : p0x + sg * D[i][0];
        const float py = j == 0 ? p0y : p0y + sg * D[i][1];
        const float pz = j == 0 ? p0z : p0z + sg * D[i][2];
        const float n2 = px * px + py * py + pz * pz;
        if (c.model == 0) {
            ok = ok && pz > 0.0f && pz * pz >= UT_COSMIN * UT_COSMIN * n2;
        } else {
            // theta <= theta_lim  <=>  p_z >= cos(theta_lim) |p|  (theta_lim < pi)
            const float nn = sqrtf(n2);
            ok = ok && nn > 0.0f && pz >= kb_c2 * nn;
        }
    }
    if (!ok) return false;
    // image offsets of the six outer points from the centre's image
    float dxs[6], dys[6], y0x, y0y;
    if (c.model == 0) {
        const float iz = 1.0f / p0z;
        y0x = c.fx * (p0x * iz) + c.cx;
        y0y = c.fy * (p0y * iz) + c.cy;
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            // u(p0 +- D) - u(p0) = +- f_x (D_x p0z - p0x D_z) / ((p0z +- D_z) p0z): no cancellation
            const float nx = D[i][0] * p0z - p0x * D[i][2], ny = D[i][1] * p0z - p0y * D[i][2];
            const float ip = 1.0f / ((p0z + D[i][2]) * p0z), im = 1.0f / ((p0z - D[i][2]) * p0z);
            dxs[2 * i] = c.fx * nx * ip;
            dys[2 * i] = c.fy * ny * ip;
            dxs[2 * i + 1] = -c.fx * nx * im;
            dys[2 * i + 1] = -c.fy * ny * im;
        }
    } else {
        const float2 y0 = ut_kb_image(c, p0x, p0y, p0z);
        y0x = y0.x + c.cx;
        y0y = y0.y + c.cy;
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            const float2 a = ut_kb_image(c, p0x + D[i][0], p0y + D[i][1], p0z + D[i][2]);
            const float2 b = ut_kb_image(c, p0x - D[i][0], p0y - D[i][1], p0z - D[i][2]);
            dxs[2 * i] = a.x - y0.x;
            dys[2 * i] = a.y - y0.y;
            dxs[2 * i + 1] = b.x - y0.x;
            dys[2 * i + 1] = b.y - y0.y;
        }
    }
    // mean (weights 1/6 on the outer points, 0 on the centre) and covariance
    // 2 (0 - mbar)(0 - mbar)^T + sum_j (1/6)(d_j - mbar)(d_j - mbar)^T = (1/6) sum_j d_j d_j^T + mbar mbar^T
    float mx = 0.f, my = 0.f, sxx = 0.f, sxy = 0.f, syy = 0.f;
#pragma unroll
    for (int j = 0; j < 6; ++j) {
        mx += dxs[j];
        my += dys[j];
        sxx += dxs[j] * dxs[j];
        sxy += dxs[j] * dys[j];
        syy += dys[j] * dys[j];
    }
    mx *= (1.0f / 6.0f);
    my *= (1.0f / 6.0f);
    sxx = sxx * (1.0f / 6.0f) + mx * mx + UT_VLP;
    sxy = sxy * (1.0f / 6.0f) + mx * my;
    syy = syy * (1.0f / 6.0f) + my * my + UT_VLP;
    const float idet = 1.0f / (sxx * syy - sxy * sxy);
    const float k2 = 2.0f * logf(255.0f * ua.sig_eff[gid]);
    e[0] = y0x + mx;
    e[1] = y0y + my;
    e[2] = syy * idet;
    e[3] = -sxy * idet;
    e[4] = sxx * idet;
    q = make_float4(k2, -e[3] / e[4], -e[3] / e[2], 0.0f);
    if (!(k2 > 0.0f)) {
        tx0 = ty0 = 0;
        tx1 = ty1 = -1;
        return true;
    }
    // tiles whose pixel-centre rectangle [8 t + 1/2, 8 t + 15/2] meets the ellipse's
    // bounding box (widened by far more than its FP32 error; the test decides)
    const float hx = sqrtf(k2 * sxx), hy = sqrtf(k2 * syy);
    const float gx = 0.01f + 1e-3f * hx, gy = 0.01f + 1e-3f * hy;
    const float lim = 1e8f;
    tx0 = max((int)ceilf(fmaxf((e[0] - hx - gx - (TILE - 0.5f)) / TILE, -lim)), 0);
    tx1 = min((int)floorf(fminf((e[0] + hx + gx - 0.5f) / TILE, lim)), c.tiles_x - 1);
    ty0 = max((int)ceilf(fmaxf((e[1] - hy - gy - (TILE - 0.5f)) / TILE, -lim)), 0);
    ty1 = min((int)floorf(fminf((e[1] + hy + gy - 0.5f) / TILE, lim)), c.tiles_y - 1);
    return true;
}

// Candidate tiles of a silhouette ellipse e (centre, A, B, C, threshold): the
// tiles whose pixel-centre rectangle meets the ellipse's bounding box, widened
// by the test's rectangle growth and by 5% (det = AC - B^2 loses up to ~2.5% to
// cancellation at the largest aspect the rule accepts, 1000).  The half-widths
// of {Q <= t} are sqrt(t C / det) and sqrt(t A / det).
__device__ __forceinline__ void ellipse_tile_box(const CamParams &c, const float *e, int &tx0, int &tx1, int &ty0,
                                                 int &ty1) {
    const float det = e[2] * e[4] - e[3] * e[3];
    const float hx = sqrtf(fmaxf(e[5] * e[4] / det, 0.0f)) * 1.05f + ELL_GROW + 0.01f;
    const float hy = sqrtf(fmaxf(e[5] * e[2] / det, 0.0f)) * 1.05f + ELL_GROW + 0.01f;
    const float lim = 1e8f;
    tx0 = max((int)ceilf(fmaxf((e[0] - hx - (TILE - 0.5f)) / TILE, -lim)), 0);
    tx1 = min((int)floorf(fminf((e[0] + hx - 0.5f) / TILE, lim)), c.tiles_x - 1);
    ty0 = max((int)ceilf(fmaxf((e[1] - hy - (TILE - 0.5f)) / TILE, -lim)), 0);
    ty1 = min((int)floorf(fminf((e[1] + hy - 0.5f) / TILE, lim)), c.tiles_y - 1);
}

// Count (MODE 0) and emit (MODE 1) of the (tile, Gaussian) pairs.
//
// Each lane prepares one Gaussian (slot): flag, rule record, direction, cone,
// silhouette record, candidate box.  The warp then walks the concatenation of
// its 32 slots' candidate tiles 32 at a time, each lane testing one (slot,
// tile) candidate with the prefilter and the rule's two tests, so lanes stay
// busy whether a Gaussian covers one tile or hundreds.  A slot's passes in an iteration are a
// contiguous run of the ballot, which its owner lane folds into its count and,
// for boxes of at most 256 tiles, into a 256-bit pass mask kept in the cache
// (3 uint4 per Gaussian: box, mask) between the two passes.  MODE 1 (slots =
// Gaussians in depth order) expands a cached slot's set bits only (no rule
// evaluation) and writes pairs at offsets[pos] + rank.  Boxes over PACK_MAX
// tiles walk their box with the whole warp; those over MASK_MAX tiles reserve
// box-size room in a list buffer (atomic cursor; when it is full the emit pass
// evaluates the rule again) and the count pass writes their passing tile ids
// there, which the emit pass copies.  Gaussians without a box (a cone too
// wide, or reaching a fisheye's rim) take the super-tile walk.
constexpr uint32_t NO_CACHE = 0xffffffffu;
constexpr int BIN_WARPS = 8;
constexpr uint32_t PACK_MAX = 96;      // slots with more candidates walk their box with the whole warp
constexpr uint32_t MASK_MAX = 256;     // boxes up to this many tiles keep their pass mask
constexpr uint32_t CACHE_MASK = 0u, CACHE_LIST = 1u;   // cache header .w (NO_CACHE: nothing kept)

// OR a 32-bit chunk of pass bits into the 256-bit mask m at bit offset at.
__device__ __forceinline__ void mask_or(uint32_t m[8], uint32_t bits, uint32_t at) {
    const uint32_t wi = at >> 5, sh = at & 31u;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        if ((uint32_t)q == wi) m[q] |= bits << sh;
        if (sh != 0u && (uint32_t)q == wi + 1u) m[q] |= bits >> (32u - sh);
    }
}

// Super-tile walk for one Gaussian by the whole warp; returns its pair count.
// ell: the slot's silhouette ellipse (ELL_F floats 32 apart, in shared memory), or nullptr.
template <int MODE>
__device__ __forceinline__ uint32_t bin_walk_supers(const CamParams &c, const float *g, const float4 gv,
                                                    const float2 half, const float *__restrict__ table,
                                                    const float *__restrict__ super, float mzf, uint32_t gid,
                                                    uint32_t base, uint32_t *__restrict__ out_tile,
                                                    uint32_t *__restrict__ out_gid, const float *ell,
                                                    const float2 lo) {
    const int lane = threadIdx.x & 31;
    const int nsup = c.supers_x * c.supers_y;
    uint32_t cnt = 0;
    for (int s0 = 0; s0 < nsup; s0 += 32) {
        const int s = s0 + lane;
        bool sp = false;
        if (s < nsup) sp = cone_prefilter(gv, half, super + 6 * (size_t)s);
        uint32_t bal = __ballot_sync(0xffffffffu, sp);
        while (bal) {
            const int b = __ffs(bal) - 1;
            bal &= bal - 1;
            const int ss = s0 + b;
            const int sx = ss % c.supers_x, sy = ss / c.supers_x;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int child = lane + 32 * h;
                const int tx = sx * SUPER + (child % SUPER), ty = sy * SUPER + (child / SUPER);
                bool tp = false;
                uint32_t tile = 0;
                if (tx < c.tiles_x && ty < c.tiles_y) {
                    tile = (uint32_t)(ty * c.tiles_x + tx);
                    float tt[6];
                    tile_record(table, tile, mzf, tt);
                    if (cone_prefilter(gv, half, tt)) {
                        const int f = rule_pass_lo(lo.x, lo.y, gv, tt) ? 1 : rule_test_fast(g, gv, tt);
                        tp = f == 2 ? rule_test(g, gv, tt) : f == 1;
                    }
                    if (tp && ell) tp = ell_keep<32>(c, ell, gv, tt, tx, ty);
                }
                const uint32_t tb = __ballot_sync(0xffffffffu, tp);
                if (MODE == 1 && tp) {
                    const uint32_t pos = base + cnt + __popc(tb & ((1u << lane) - 1u));
                    out_tile[pos] = tile;
                    out_gid[pos] = gid;
                }
                cnt += __popc(tb);
            }
        }
    }
    return cnt;
}

// Candidate box of one Gaussian walked by the whole warp; returns its pair count
// and (boxes of at most MASK_MAX tiles) its pass mask in m (same on every lane).
// ut: the slot is a UT ellipse (g[0..4] = ybar, A, B, C; gv = k^2, -B/C, -B/A).
template <int MODE, bool UT>
__device__ __forceinline__ uint32_t bin_walk_box(const CamParams &c, const float *g, const float4 gv,
                                                 const float2 half, const float *__restrict__ table, float mzf,
                                                 int tx0, int ty0, int bw, uint32_t nb, uint32_t gid, uint32_t base,
                                                 uint32_t m[8], uint32_t *__restrict__ list,
                                                 uint32_t *__restrict__ out_tile, uint32_t *__restrict__ out_gid,
                                                 bool ut, const float *ell, const float2 lo) {
    const int lane = threadIdx.x & 31;
    uint32_t cnt = 0;
    int qy = 0, qx = lane;                     // candidate k0 + lane = qy * bw + qx
    while (qx >= bw) {
        qx -= bw;
        ++qy;
    }
    const int sy = 32 / bw, sx = 32 % bw;      // advance by 32 candidates
    for (uint32_t k0 = 0; k0 < nb; k0 += 32) {
        bool tp = false;
        uint32_t tile = 0;
        if (k0 + (uint32_t)lane < nb) {
            tile = (uint32_t)((ty0 + qy) * c.tiles_x + tx0 + qx);
            if (UT && ut) {
                tp = ellipse_rect_test(c, g, gv, tx0 + qx, ty0 + qy, 0.0f);
            } else {
                float tt[6];
                tile_record(table, tile, mzf, tt);
                if (cone_prefilter(gv, half, tt)) {
                    const int f = rule_pass_lo(lo.x, lo.y, gv, tt) ? 1 : rule_test_fast(g, gv, tt);
                    tp = f == 2 ? rule_test(g, gv, tt) : f == 1;
                }
                if (tp && ell) tp = ell_keep<32>(c, ell, gv, tt, tx0 + qx, ty0 + qy);
            }
        }
        const uint32_t tb = __ballot_sync(0xffffffffu, tp);
        if (MODE == 1 && tp) {
            const uint32_t pos = base + cnt + __popc(tb & ((1u << lane) - 1u));
            out_tile[pos] = tile;
            out_gid[pos] = gid;
        }
        if (MODE == 0 && list && tp) list[cnt + __popc(tb & ((1u << lane) - 1u))] = tile;
        if (MODE == 0 && nb <= MASK_MAX) {
#pragma unroll
            for (int q = 0; q < 8; ++q)
                if ((uint32_t)q == (k0 >> 5)) m[q] = tb;
        }
        cnt += __popc(tb);
        qy += sy;
        qx += sx;
        if (qx >= bw) {
            qx -= bw;
            ++qy;
        }
    }
    return cnt;
}

template <int MODE, bool UT>
__global__ void __launch_bounds__(32 * BIN_WARPS, 4) bin_kernel(CamParams c, GaussArgs ua,
                                                                const float *__restrict__ binrec,
                                                                const float4 *__restrict__ gview,
                                                                const float2 *__restrict__ gcone,
                                                                const uint8_t *__restrict__ gflag,
                                                                const float *__restrict__ table,
                                                                const float *__restrict__ super,
                                                                const float *__restrict__ mcam, float mzf,
                                                                int64_t n,
                                                                const uint32_t *__restrict__ order,
                                                                const uint32_t *__restrict__ offsets,
                                                                uint32_t *__restrict__ counts,
                                                                uint4 *__restrict__ cache,
                                                                uint32_t *__restrict__ blist,
                                                                unsigned long long *__restrict__ bcursor,
                                                                unsigned long long bcap,
                                                                uint32_t *__restrict__ out_tile,
                                                                uint32_t *__restrict__ out_gid) {
    __shared__ float s_g[BIN_WARPS][5][32];        // kap, ks, kr, r1sq, s2 (flag is 1 for boxed slots)
    __shared__ float4 s_gv[BIN_WARPS][32];
    __shared__ float2 s_half[BIN_WARPS][32];
    __shared__ float2 s_lo[BIN_WARPS][32];         // rule_pass_lo's cone at the view's smallest m
    __shared__ int4 s_box[BIN_WARPS][32];          // tx0, ty0, box width, bits: cached (1), UT (2), silhouette (4)
    __shared__ float s_inv[BIN_WARPS][32];         // 1 / box width
    __shared__ uint4 s_mask[BIN_WARPS][2][32];     // MODE 1: cached pass mask (8 words)
    __shared__ float s_ell[BIN_WARPS][ELL_F][32];  // silhouette ellipse (valid: s_box .w bit 4)
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int64_t pos = ((int64_t)blockIdx.x * BIN_WARPS + wid) * 32 + lane;
    const bool have = pos < n;
    const uint32_t gid = have ? (MODE == 0 ? (uint32_t)pos : order[pos]) : 0u;
    const uint32_t base = (MODE == 1 && have) ? offsets[pos] : 0u;
    // ---- slot set-up
    uint32_t nb = 0, fl = 0, npk = 0, lofs = 0, lcnt = 0;
    bool walk = false, cached = false, big = false, listed = false, utslot = false, ellv = false;
    float4 el0 = make_float4(0.f, 0.f, 0.f, 0.f), el1 = el0, el2 = el0;   // silhouette record
    float g[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    float4 gv = make_float4(0.f, 0.f, 0.f, 0.f);
    float2 half = make_float2(0.f, 1.f);
    float2 lo2 = make_float2(RULE_NONE, 0.f);
    int tx0 = 0, tx1 = -1, ty0 = 0, ty1 = -1;
    if (have) {
        fl = gflag[gid];
        if (MODE == 1) {
            const uint4 cc = cache[3 * (size_t)gid];
            if (cc.w == CACHE_LIST) {
                listed = true;
                lofs = cc.x;
                lcnt = cc.y;
            } else if (UT && cc.w == CACHE_UT) {
                // a UT slot whose tiles are tested again: box and ellipse from the count pass
                utslot = true;
                tx0 = (int)(cc.x & 0xffffu);
                ty0 = (int)(cc.x >> 16);
                tx1 = (int)(cc.y & 0xffffu);
                ty1 = (int)(cc.y >> 16);
                const uint4 e0 = cache[3 * (size_t)gid + 1], e1 = cache[3 * (size_t)gid + 2];
                g[0] = __uint_as_float(e0.x); g[1] = __uint_as_float(e0.y); g[2] = __uint_as_float(e0.z);
                g[3] = __uint_as_float(e0.w); g[4] = __uint_as_float(e1.x);
                g[5] = 3.0f;
                gv = make_float4(__uint_as_float(e1.y), __uint_as_float(e1.z), __uint_as_float(e1.w), 0.0f);
                nb = (uint32_t)(tx1 - tx0 + 1) * (uint32_t)(ty1 - ty0 + 1);
                big = nb > PACK_MAX;
                npk = big ? 0u : nb;
            } else if (cc.w == CACHE_MASK) {
                cached = true;
                tx0 = (int)(cc.x & 0xffffu);
                ty0 = (int)(cc.x >> 16);
                tx1 = tx0 + (int)(cc.y & 0xffffu) - 1;
                nb = cc.y >> 16;
                const uint4 m0 = cache[3 * (size_t)gid + 1], m1 = cache[3 * (size_t)gid + 2];
                s_mask[wid][0][lane] = m0;
                s_mask[wid][1][lane] = m1;
                npk = (uint32_t)(__popc(m0.x) + __popc(m0.y) + __popc(m0.z) + __popc(m0.w) + __popc(m1.x) +
                                 __popc(m1.y) + __popc(m1.z) + __popc(m1.w));
            }
        }
        if (MODE == 0 && UT && fl == 1) {
            float4 uq;
            if (ut_ellipse(c, ua, gid, g, uq, tx0, tx1, ty0, ty1)) {
                utslot = true;
                g[5] = 3.0f;
                gv = uq;
                const int bw = tx1 - tx0 + 1, bh = ty1 - ty0 + 1;
                nb = (bw > 0 && bh > 0) ? (uint32_t)(bw * bh) : 0u;
                big = nb > PACK_MAX;
                npk = big ? 0u : nb;
            }
        }
        if (fl != 0 && !cached && !listed && !utslot) {
#pragma unroll
            for (int k = 0; k < 5; ++k) g[k] = binrec[BINREC * (size_t)gid + k];
            g[5] = (float)fl;
            gv = gview[gid];
            half = gcone[gid];
            lo2 = rule_lo(g, gv.w, fmaxf(mcam[MCAM_MMIN], mzf));
            if (fl == 1) {
                // silhouette record of the rule's bounding ellipsoid (from the view records)
                el0 = ua.ell[3 * (size_t)gid];
                el1 = ua.ell[3 * (size_t)gid + 1];
                el2 = ua.ell[3 * (size_t)gid + 2];
                ellv = el1.y > 0.0f;
            }
            bool boxed =
                fl == 1 && half.y >= 1e-3f &&
                (c.model == 0 ? pinhole_tile_box(c, gv, half, mcam[1], tx0, tx1, ty0, ty1)
                              : kb_tile_box(c, gv, half, mcam, tx0, tx1, ty0, ty1));
            if (ellv && c.model == 0) {
                // every tile the silhouette test keeps lies in the ellipse's box
                int ex0, ex1, ey0, ey1;
                const float eb[6] = {el0.x, el0.y, el0.z, el0.w, el1.x, el1.y};
                ellipse_tile_box(c, eb, ex0, ex1, ey0, ey1);
                if (boxed) {
                    tx0 = max(tx0, ex0); tx1 = min(tx1, ex1);
                    ty0 = max(ty0, ey0); ty1 = min(ty1, ey1);
                } else {
                    tx0 = ex0; tx1 = ex1; ty0 = ey0; ty1 = ey1;
                    boxed = true;
                }
            }
            if (boxed) {
                const int bw = tx1 - tx0 + 1, bh = ty1 - ty0 + 1;
                nb = (bw > 0 && bh > 0) ? (uint32_t)(bw * bh) : 0u;
                big = nb > PACK_MAX;
                npk = big ? 0u : nb;
            } else {
                walk = true;                     // pass-all (flag 2) or unbounded cone
            }
        }
    }
    s_g[wid][0][lane] = g[0]; s_g[wid][1][lane] = g[1]; s_g[wid][2][lane] = g[2];
    s_g[wid][3][lane] = g[3]; s_g[wid][4][lane] = g[4];
    s_gv[wid][lane] = gv;
    s_half[wid][lane] = half;
    s_lo[wid][lane] = lo2;
    s_box[wid][lane] = make_int4(tx0, ty0, tx1 - tx0 + 1, (cached ? 1 : 0) | (utslot ? 2 : 0) | (ellv ? 4 : 0));
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        s_ell[wid][k][lane] = k == 0 ? el0.x : k == 1 ? el0.y : k == 2 ? el0.z : el0.w;
        s_ell[wid][4 + k][lane] = k == 0 ? el1.x : k == 1 ? el1.y : k == 2 ? el1.z : el1.w;
        s_ell[wid][8 + k][lane] = k == 0 ? el2.x : k == 1 ? el2.y : k == 2 ? el2.z : el2.w;
    }
    s_inv[wid][lane] = tx1 >= tx0 ? 1.0f / (float)(tx1 - tx0 + 1) : 0.0f;
    // exclusive prefix of the packed slots' candidate counts (a cached slot of the emit
    // pass contributes its passing candidates only; big boxes are walked below)
    uint32_t start = npk;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, start, o);
        if (lane >= o) start += y;
    }
    const uint32_t total = __shfl_sync(0xffffffffu, start, 31);
    start -= npk;
    __syncwarp();
    // ---- packed walk over the candidates of the 32 slots
    uint32_t cnt = 0;
    uint32_t pm[8] = {0u, 0u, 0u, 0u, 0u, 0u, 0u, 0u};
    for (uint32_t it0 = 0; it0 < total; it0 += 32) {
        const uint32_t p = it0 + (uint32_t)lane;
        // owner slot of candidate p: the last lane whose start is <= p (all lanes search)
        int sl = 0;
#pragma unroll
        for (int step = 16; step > 0; step >>= 1) {
            const int cand = sl + step;
            const uint32_t sv = __shfl_sync(0xffffffffu, start, cand & 31);
            if (cand < 32 && sv <= p) sl = cand;
        }
        const uint32_t sstart = __shfl_sync(0xffffffffu, start, sl);
        bool tp = false;
        uint32_t tile = 0u;
        if (p < total) {
            uint32_t k = p - sstart;
            const int4 bx = s_box[wid][sl];
            if (MODE == 1 && (bx.w & 1)) {
                // the k-th passing candidate of a cached slot: the (k+1)-th set bit of its mask
                const uint4 m0 = s_mask[wid][0][sl], m1 = s_mask[wid][1][sl];
                const uint32_t mw[8] = {m0.x, m0.y, m0.z, m0.w, m1.x, m1.y, m1.z, m1.w};
                uint32_t rem = k, bit = 0;
                bool found = false;
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    const uint32_t pc = (uint32_t)__popc(mw[q]);
                    if (!found && rem < pc) {
                        bit = 32u * q + __fns(mw[q], 0u, (int)rem + 1);
                        found = true;
                    }
                    if (!found) rem -= pc;
                }
                k = bit;
                tp = true;
            }
            // k = ky * width + kx, from a float reciprocal corrected to the exact quotient
            int ky = (int)((float)k * s_inv[wid][sl]);
            int kx = (int)k - ky * bx.z;
            if (kx < 0) {
                --ky;
                kx += bx.z;
            } else if (kx >= bx.z) {
                ++ky;
                kx -= bx.z;
            }
            tile = (uint32_t)((bx.y + ky) * c.tiles_x + bx.x + kx);
            if (!(MODE == 1 && (bx.w & 1))) {
                const float gg[6] = {s_g[wid][0][sl], s_g[wid][1][sl], s_g[wid][2][sl], s_g[wid][3][sl],
                                     s_g[wid][4][sl], 1.0f};
                const float4 sgv = s_gv[wid][sl];
                if (UT && (bx.w & 2)) {
                    tp = ellipse_rect_test(c, gg, sgv, bx.x + kx, bx.y + ky, 0.0f);
                } else {
                    float tt[6];
                    tile_record(table, tile, mzf, tt);
                    if (cone_prefilter(sgv, s_half[wid][sl], tt)) {
                        const float2 lo = s_lo[wid][sl];
                        const int f = rule_pass_lo(lo.x, lo.y, sgv, tt) ? 1 : rule_test_fast(gg, sgv, tt);
                        tp = f == 2 ? rule_test(gg, sgv, tt) : f == 1;
                    }
                    if (tp && (bx.w & 4)) tp = ell_keep<32>(c, &s_ell[wid][0][sl], sgv, tt, bx.x + kx, bx.y + ky);
                }
            }
        }
        const uint32_t bal = __ballot_sync(0xffffffffu, tp);
        // this slot's candidates in the iteration: lanes [lo, hi)
        const uint32_t lo32 = start > it0 ? start - it0 : 0u;
        const uint32_t hi32 = start + npk > it0 ? min(start + npk - it0, 32u) : 0u;
        uint32_t mine = 0u;
        if (lo32 < hi32) {
            const uint32_t width = hi32 - lo32;
            mine = (width == 32u ? bal : (bal >> lo32) & ((1u << width) - 1u));
        }
        if (MODE == 1) {
            // rank among the owner's passing candidates so far (every lane takes part)
            const uint32_t ocnt = __shfl_sync(0xffffffffu, cnt, sl);
            const uint32_t obase = __shfl_sync(0xffffffffu, base, sl);
            const uint32_t olo = __shfl_sync(0xffffffffu, lo32, sl);
            const uint32_t ogid = __shfl_sync(0xffffffffu, gid, sl);
            if (tp) {
                const uint32_t below = bal & ((1u << lane) - 1u) & ~((1u << olo) - 1u);
                const uint32_t dst = obase + ocnt + (uint32_t)__popc(below);
                out_tile[dst] = tile;
                out_gid[dst] = ogid;
            }
        }
        __syncwarp();
        if (MODE == 0 && lo32 < hi32) mask_or(pm, mine, it0 + lo32 - start);
        cnt += (uint32_t)__popc(mine);
    }
    // ---- big boxes: one slot at a time by the whole warp
    uint32_t bb = __ballot_sync(0xffffffffu, big);
    while (bb) {
        const int sl = __ffs(bb) - 1;
        bb &= bb - 1;
        float gg[6];
#pragma unroll
        for (int k = 0; k < 6; ++k) gg[k] = __shfl_sync(0xffffffffu, g[k], sl);
        float4 sgv;
        sgv.x = __shfl_sync(0xffffffffu, gv.x, sl); sgv.y = __shfl_sync(0xffffffffu, gv.y, sl);
        sgv.z = __shfl_sync(0xffffffffu, gv.z, sl); sgv.w = __shfl_sync(0xffffffffu, gv.w, sl);
        float2 sh;
        sh.x = __shfl_sync(0xffffffffu, half.x, sl); sh.y = __shfl_sync(0xffffffffu, half.y, sl);
        const int btx0 = __shfl_sync(0xffffffffu, tx0, sl), bty0 = __shfl_sync(0xffffffffu, ty0, sl);
        const int bw = __shfl_sync(0xffffffffu, tx1, sl) - btx0 + 1;
        const uint32_t bnb = __shfl_sync(0xffffffffu, nb, sl);
        const uint32_t sgid = __shfl_sync(0xffffffffu, gid, sl);
        const uint32_t sbase = __shfl_sync(0xffffffffu, base, sl);
        uint32_t wm[8] = {0u, 0u, 0u, 0u, 0u, 0u, 0u, 0u};
        uint32_t *lst = nullptr;
        unsigned long long lo = 0ull;
        if (MODE == 0 && bnb > MASK_MAX) {
            if (lane == 0) lo = atomicAdd(bcursor, (unsigned long long)bnb);
            lo = __shfl_sync(0xffffffffu, lo, 0);
            if (lo + bnb <= bcap) lst = blist + lo;
        }
        const float *sel = &s_ell[wid][0][sl];
        const bool sev = (s_box[wid][sl].w & 4) != 0;
        const uint32_t wc = bin_walk_box<MODE, UT>(c, gg, sgv, sh, table, mzf, btx0, bty0, bw, bnb, sgid, sbase,
                                                   wm, lst, out_tile, out_gid, gg[5] == 3.0f, sev ? sel : nullptr,
                                                   s_lo[wid][sl]);
        if (lane == sl) {
            cnt = wc;
#pragma unroll
            for (int q = 0; q < 8; ++q) pm[q] = wm[q];
            listed = lst != nullptr;
            lofs = (uint32_t)lo;
        }
    }
    // ---- emit of list-cached slots: copy the kept tile ids, one slot at a time by the whole warp
    if (MODE == 1) {
        uint32_t lb = __ballot_sync(0xffffffffu, listed);
        while (lb) {
            const int sl = __ffs(lb) - 1;
            lb &= lb - 1;
            const uint32_t o = __shfl_sync(0xffffffffu, lofs, sl), nc = __shfl_sync(0xffffffffu, lcnt, sl);
            const uint32_t sgid = __shfl_sync(0xffffffffu, gid, sl), sbase = __shfl_sync(0xffffffffu, base, sl);
            for (uint32_t k = (uint32_t)lane; k < nc; k += 32) {
                out_tile[sbase + k] = blist[o + k];
                out_gid[sbase + k] = sgid;
            }
        }
    }
    // ---- slots without a box: the super-tile walk, one slot at a time by the whole warp
    uint32_t wb = __ballot_sync(0xffffffffu, walk);
    while (wb) {
        const int sl = __ffs(wb) - 1;
        wb &= wb - 1;
        float gg[6];
#pragma unroll
        for (int k = 0; k < 6; ++k) gg[k] = __shfl_sync(0xffffffffu, g[k], sl);
        float4 sgv;
        sgv.x = __shfl_sync(0xffffffffu, gv.x, sl); sgv.y = __shfl_sync(0xffffffffu, gv.y, sl);
        sgv.z = __shfl_sync(0xffffffffu, gv.z, sl); sgv.w = __shfl_sync(0xffffffffu, gv.w, sl);
        float2 sh;
        sh.x = __shfl_sync(0xffffffffu, half.x, sl); sh.y = __shfl_sync(0xffffffffu, half.y, sl);
        const uint32_t sgid = __shfl_sync(0xffffffffu, gid, sl);
        const uint32_t sbase = __shfl_sync(0xffffffffu, base, sl);
        const float *sel = &s_ell[wid][0][sl];
        const bool sev = (s_box[wid][sl].w & 4) != 0;
        const uint32_t wc = bin_walk_supers<MODE>(c, gg, sgv, sh, table, super, mzf, sgid, sbase, out_tile, out_gid,
                                                  sev ? sel : nullptr, s_lo[wid][sl]);
        if (lane == sl) cnt = wc;
    }
    if (MODE == 0 && have) {
        counts[gid] = cnt;
        if (fl != 0 && !walk && nb <= MASK_MAX) {
            cache[3 * (size_t)gid] = make_uint4((uint32_t)tx0 | ((uint32_t)ty0 << 16),
                                                (uint32_t)(tx1 - tx0 + 1) | (nb << 16), 0u, CACHE_MASK);
            cache[3 * (size_t)gid + 1] = make_uint4(pm[0], pm[1], pm[2], pm[3]);
            cache[3 * (size_t)gid + 2] = make_uint4(pm[4], pm[5], pm[6], pm[7]);
        } else if (listed) {
            cache[3 * (size_t)gid] = make_uint4(lofs, cnt, 0u, CACHE_LIST);
        } else if (UT && utslot) {
            cache[3 * (size_t)gid] = make_uint4((uint32_t)tx0 | ((uint32_t)ty0 << 16),
                                                (uint32_t)tx1 | ((uint32_t)ty1 << 16), 0u, CACHE_UT);
            cache[3 * (size_t)gid + 1] = make_uint4(__float_as_uint(g[0]), __float_as_uint(g[1]),
                                                    __float_as_uint(g[2]), __float_as_uint(g[3]));
            cache[3 * (size_t)gid + 2] = make_uint4(__float_as_uint(g[4]), __float_as_uint(gv.x),
                                                    __float_as_uint(gv.y), __float_as_uint(gv.z));
        } else {
            cache[3 * (size_t)gid] = make_uint4(0u, 0u, 0u, NO_CACHE);
        }
    }
}

// ---------------------------------------------------------------- launchers

cudaError_t launch_tile_tables(const CamParams &c, float *table, float *super, float *mcam, cudaStream_t s) {
    const int nt = c.tiles_x * c.tiles_y, ns = c.supers_x * c.supers_y;
    if (nt == 0) return cudaSuccess;
    tile_table_kernel<<<nt, TILE_PX, 0, s>>>(c, table);
    note_launches(1);
    super_table_kernel<<<(unsigned)div_up(ns, 128), 128, 0, s>>>(c, table, super);
    note_launches(1);
    max_m_kernel<<<1, 1024, 0, s>>>(c, table, nt, mcam);
    note_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_gauss_scene_rule(const SceneParams &sp, float *binrec, cudaStream_t s) {
    if (sp.n == 0) return cudaSuccess;
    gauss_scene_rule_kernel<<<(unsigned)div_up(sp.n, 256), 256, 0, s>>>(sp, binrec);
    note_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_gauss_view_rule(const CamParams &c, const SceneParams &sp, float4 *gview, uint8_t *gflag,
                                   cudaStream_t s) {
    if (sp.n == 0) return cudaSuccess;
    gauss_view_rule_kernel<<<(unsigned)div_up(sp.n, 256), 256, 0, s>>>(c, sp, gview, gflag);
    note_launches(1);
    return cudaGetLastError();
}

// gell: silhouette ellipses from the view records; ut_means/ut_W/ut_sig_eff non-null: UT binning.
cudaError_t launch_bin_count(const CamParams &c, const float *binrec, const float4 *gview, const float2 *gcone,
                             const uint8_t *gflag, const float *table, const float *super, const float *mcam,
                             float mzf, int64_t n, uint32_t *counts, uint4 *cache, uint32_t *blist,
                             unsigned long long *bcursor, unsigned long long bcap, const float4 *gell,
                             const float *ut_means, const float *ut_W, const float *ut_sig_eff, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    const GaussArgs ua{gell, ut_means, ut_W, ut_sig_eff};
    const unsigned grid = (unsigned)div_up(n, 32 * BIN_WARPS);
    if (ut_W)
        bin_kernel<0, true><<<grid, 32 * BIN_WARPS, 0, s>>>(c, ua, binrec, gview, gcone, gflag, table, super, mcam,
                                                           mzf, n, nullptr, nullptr, counts, cache, blist, bcursor,
                                                           bcap, nullptr, nullptr);
    else
        bin_kernel<0, false><<<grid, 32 * BIN_WARPS, 0, s>>>(c, ua, binrec, gview, gcone, gflag, table, super, mcam,
                                                            mzf, n, nullptr, nullptr, counts, cache, blist, bcursor,
                                                            bcap, nullptr, nullptr);
    note_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_bin_emit(const CamParams &c, const float *binrec, const float4 *gview, const float2 *gcone,
                            const uint8_t *gflag, const float *table, const float *super, const float *mcam,
                            float mzf, int64_t n_sorted, const uint32_t *order, const uint32_t *offsets,
                            const uint4 *cache, const uint32_t *blist, uint32_t *out_tile, uint32_t *out_gid,
                            const float4 *gell, bool ut, cudaStream_t s) {
    if (n_sorted == 0) return cudaSuccess;
    const GaussArgs ua{gell, nullptr, nullptr, nullptr};
    const unsigned grid = (unsigned)div_up(n_sorted, 32 * BIN_WARPS);
    if (ut)
        bin_kernel<1, true><<<grid, 32 * BIN_WARPS, 0, s>>>(c, ua, binrec, gview, gcone, gflag, table, super, mcam,
                                                           mzf, n_sorted, order, offsets, nullptr,
                                                           const_cast<uint4 *>(cache), const_cast<uint32_t *>(blist),
                                                           nullptr, 0ull, out_tile, out_gid);
    else
        bin_kernel<1, false><<<grid, 32 * BIN_WARPS, 0, s>>>(c, ua, binrec, gview, gcone, gflag, table, super, mcam,
                                                            mzf, n_sorted, order, offsets, nullptr,
                                                            const_cast<uint4 *>(cache),
                                                            const_cast<uint32_t *>(blist), nullptr, 0ull, out_tile,
                                                            out_gid);
    note_launches(1);
    return cudaGetLastError();
}

}  // namespace conegs
