// K6/K7: adjoint of the render (reverse-mode, hand written).
//
// K6 walks each tile's list back to front for every pixel, recovering the
// transmittance before each contributing pair by division from the final T
// kept by the forward pass (T_k = T_{k+1} / (1 - a_k)); no per-pair state is
// stored by the forward.  Each pair's response is recomputed with the same
// code as the forward (so the same pairs pass the alpha and stop tests) and
// differentiated.  For C = sum_k c_k a_k T_k and T_fin = prod_k (1 - a_k):
//   dL/dc_k = a_k T_k dL/dC
//   dL/da_k = T_k c_k.dL/dC - (S_k.dL/dC + T_fin dL/dT_fin)/(1 - a_k),
//   S_k = sum_{j>k} c_j a_j T_j (colour behind k)                    (Eq. 4)
// and da/dT = 1 below the 0.99 clamp.  As in the forward pass, a broadcast
// cone pre-test builds each lane's mask of the staged entries it reached,
// then lanes walk their own passing entries back to front in lockstep; each
// pair's gradient w.r.t. the view record (W_eff 9, o_u 3, sigma_eff, rgb 3)
// is added to a per-Gaussian buffer with four float4 atomics (lanes of a warp
// often hold the same entry at once, which rules out shared-memory sums).
// K7 applies the chain rule from the record to the scene parameters:
// o_u = W (o - mu), W_ab = R_ba / s_eff,a, s_eff = sqrt(s^2 + rho^2),
// sigma_eff = sigma prod s/s_eff (Eq. 10), s = exp(log s),
// sigma = sigmoid(logit), R = R(q/|q|), rgb = max(0, SH(u) + 1/2),
// u = (mu - o)/|mu - o|.  rho^2 is not differentiated.
#include "adjoint.cuh"
#include "raster.cuh"
#include "sh.cuh"

namespace conegs {

// One CTA per tile (FIRST: a tile's whole list, or the first segment of a split
// list) or per later segment of a split list.  A segment is walked back to
// front from the state the forward's suffix pass left: T after the segment and
// the colour composited behind it; pixels whose walk ended before the segment
// sit out.  Ten CTAs per SM leave it 96 registers and no spills; at twelve (80
// registers) the local-memory loads of the spilled pair state stalled the walk.
template <bool FILTER, bool FIRST, bool PIX>
__global__ void __launch_bounds__(TILE_PX, 10) raster_bwd_kernel(const RasterArgs a, const SegArgs g,
                                                             const float *__restrict__ dL_drgb,
                                                             const float *__restrict__ dL_dT,
                                                             const float *__restrict__ final_T,
                                                             float *__restrict__ g_rec) {
    __shared__ float4 s_rec[REC_F4][TILE_PX];
    __shared__ uint32_t s_gid[TILE_PX];
    __shared__ uint32_t s_maxlast;
    uint2 tw;
    if (FIRST) {
        tw = make_uint2(blockIdx.x, 0u);
    } else {
        if (blockIdx.x >= *g.total) return;
        tw = g.work[blockIdx.x];
    }
    const int tile = (int)tw.x;
    const uint32_t nseg = g.nseg[tile];
    const int tx = tile % a.tiles_x, ty = tile / a.tiles_x;
    const int i = tx * TILE + (threadIdx.x % TILE), j = ty * TILE + (threadIdx.x / TILE);
    const int64_t P = (int64_t)a.W * a.H;
    const bool inside = i < a.W && j < a.H;
    const int64_t pix = (int64_t)j * a.W + i;
    const uint2 range = a.ranges[tile];
    uint32_t b0 = range.x, b1 = range.y;
    if (nseg > 1) {
        const uint32_t seg = seg_length_dev(g);
        b0 = range.x + tw.y * seg;
        b1 = min(range.y, b0 + seg);
    }
    PixelRays px;
    uint32_t last = 0;
    float T = 1.0f, Tfin = 1.0f, GC[3] = {0.f, 0.f, 0.f}, GT = 0.f, S[3] = {0.f, 0.f, 0.f};
    if (inside && a.valid[pix]) {
        bool active = true;
        Tfin = final_T[pix];
        T = Tfin;
        if (nseg > 1) {
            const size_t q = (size_t)tile * TILE_PX + threadIdx.x;
            const uint32_t reach = g.rp_end[q];
            active = reach != NO_STOP && tw.y <= reach;
            if (active) {
                const float4 st = g.seg_c[(size_t)(g.seg_off[tile] + tw.y) * TILE_PX + threadIdx.x];
                S[0] = st.x; S[1] = st.y; S[2] = st.z;
                T = st.w;
            }
        }
        if (active) {
            load_pixel(a, pix, P, px);
            last = a.last[pix];
            GC[0] = dL_drgb[pix]; GC[1] = dL_drgb[P + pix]; GC[2] = dL_drgb[2 * P + pix];
            GT = dL_dT ? dL_dT[pix] : 0.0f;
        }
    }
    // the CTA only needs the entries up to its pixels' furthest last contributor
    if (threadIdx.x == 0) s_maxlast = 0;
    __syncthreads();
    atomicMax(&s_maxlast, last);
    __syncthreads();
    const uint32_t stop = min(b1, range.x + s_maxlast);
    for (uint32_t end = stop; end > b0;) {
        const uint32_t start = end - min((uint32_t)TILE_PX, end - b0);
        const uint32_t nb = end - start;
        __syncthreads();
        if (threadIdx.x < nb) {
            const uint32_t gid = a.gids[start + threadIdx.x];
            s_gid[threadIdx.x] = gid;
            const float4 *r = a.rec + (size_t)REC_F4 * gid;
#pragma unroll
            for (int k = 0; k < REC_F4; ++k) s_rec[k][threadIdx.x] = r[k];
        }
        __syncthreads();
        // phase 1: broadcast pre-test of the staged entries this pixel reached
        unsigned long long mask = 0ull;
        if (last > 0) {
            for (int b = 0; b < (int)nb; ++b) {
                const uint32_t walk = start + b - range.x + 1;     // 1-based walk index of this entry
                if (walk > last) break;
                if (staged_pretest<PIX>(s_rec, b, px)) mask |= 1ull << b;
            }
        }
        // phase 2: lanes walk their own passing entries back to front in lockstep
        while (__any_sync(0xffffffffu, mask != 0ull)) {
            if (mask == 0ull) continue;
            const int b = 63 - __clzll((long long)mask);
            mask &= ~(1ull << b);
            const float r7x = s_rec[7][b].x;              // rho^2 (sign bit: flat)
            const float4 r3 = s_rec[3][b];
            float4 *dst = reinterpret_cast<float4 *>(g_rec + 16 * (size_t)s_gid[b]);   // 64-byte aligned
            if (rec_is_flat(r7x)) {
                // flat Gaussian: the forward's FP64 response and its derivatives
                // dT/d(record), precomputed; dL/d(record) = dL/dT dT/d(record)
                const size_t fs = a.flat_slot[start + b];
                const float Tf = a.flat_T[fs * TILE_PX + threadIdx.x];
                if (Tf < 0.0f) continue;
                const float alpha = fminf(ALPHA_MAX, Tf);
                if (alpha < ALPHA_MIN) continue;
                const float inv_m = sfu_rcp(1.0f - alpha);
                const float Tb = T * inv_m;
                const float cG = r3.x * GC[0] + r3.y * GC[1] + r3.z * GC[2];
                const float SG = S[0] * GC[0] + S[1] * GC[1] + S[2] * GC[2];
                const float galpha = Tb * cG - (SG + GT * Tfin) * inv_m;
                const float w = alpha * Tb;
                S[0] += r3.x * w; S[1] += r3.y * w; S[2] += r3.z * w;
                T = Tb;
                const float gT = Tf < ALPHA_MAX ? galpha : 0.0f;
                const float *gd = a.flat_G + fs * 13 * TILE_PX + threadIdx.x;
                atomicAdd(dst, make_float4(gT * gd[0], gT * gd[TILE_PX], gT * gd[2 * TILE_PX], gT * gd[3 * TILE_PX]));
                atomicAdd(dst + 1, make_float4(gT * gd[4 * TILE_PX], gT * gd[5 * TILE_PX], gT * gd[6 * TILE_PX],
                                               gT * gd[7 * TILE_PX]));
                atomicAdd(dst + 2, make_float4(gT * gd[8 * TILE_PX], gT * gd[9 * TILE_PX], gT * gd[10 * TILE_PX],
                                               gT * gd[11 * TILE_PX]));
                atomicAdd(dst + 3, make_float4(gT * gd[12 * TILE_PX], w * GC[0], w * GC[1], w * GC[2]));
                continue;
            }
            PairFwd f;
            float Tresp = 0.f;
            if (!pair_response<FILTER, true>(rec_f32(s_rec[0][b], s_rec[1][b], s_rec[2][b], r3.w, r7x),
                                             a.additive != 0, px, Tresp, &f))
                continue;
            const float alpha = fminf(ALPHA_MAX, Tresp);
            if (alpha < ALPHA_MIN) continue;
            const float inv_m = sfu_rcp(1.0f - alpha);
            const float Tb = T * inv_m;                     // transmittance before this pair
            const float cG = r3.x * GC[0] + r3.y * GC[1] + r3.z * GC[2];
            const float SG = S[0] * GC[0] + S[1] * GC[1] + S[2] * GC[2];
            const float galpha = Tb * cG - (SG + GT * Tfin) * inv_m;
            const float w = alpha * Tb;
            float gW[9] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f}, gou[3] = {0.f, 0.f, 0.f};
            S[0] += r3.x * w; S[1] += r3.y * w; S[2] += r3.z * w;
            T = Tb;
            const float gT = Tresp < ALPHA_MAX ? galpha : 0.0f;
            const float gsig = pair_adjoint<FILTER>(f, rec_f32(s_rec[0][b], s_rec[1][b], s_rec[2][b], r3.w, r7x), px,
                                                    gT, gW, gou);
            atomicAdd(dst, make_float4(gW[0], gW[1], gW[2], gW[3]));
            atomicAdd(dst + 1, make_float4(gW[4], gW[5], gW[6], gW[7]));
            atomicAdd(dst + 2, make_float4(gW[8], gou[0], gou[1], gou[2]));
            atomicAdd(dst + 3, make_float4(gsig, w * GC[0], w * GC[1], w * GC[2]));
        }
        end = start;
    }
}

cudaError_t launch_backward(const RasterArgs &a, int ntiles, bool filter, uint32_t *split_scratch,
                            const float *dL_drgb, const float *dL_dT, const float *final_T, float *g_rec,
                            cudaStream_t s) {
    if (ntiles == 0) return cudaSuccess;
    int64_t items = 0;
    const SegArgs g = split_args(split_scratch, ntiles, &items);
    const unsigned later = (unsigned)(items - ntiles);
    if (filter && a.pixtest) {
        raster_bwd_kernel<true, true, true><<<ntiles, TILE_PX, 0, s>>>(a, g, dL_drgb, dL_dT, final_T, g_rec);
        raster_bwd_kernel<true, false, true><<<later, TILE_PX, 0, s>>>(a, g, dL_drgb, dL_dT, final_T, g_rec);
    } else if (filter) {
        raster_bwd_kernel<true, true, false><<<ntiles, TILE_PX, 0, s>>>(a, g, dL_drgb, dL_dT, final_T, g_rec);
        raster_bwd_kernel<true, false, false><<<later, TILE_PX, 0, s>>>(a, g, dL_drgb, dL_dT, final_T, g_rec);
    } else if (a.pixtest) {
        raster_bwd_kernel<false, true, true><<<ntiles, TILE_PX, 0, s>>>(a, g, dL_drgb, dL_dT, final_T, g_rec);
        raster_bwd_kernel<false, false, true><<<later, TILE_PX, 0, s>>>(a, g, dL_drgb, dL_dT, final_T, g_rec);
    } else {
        raster_bwd_kernel<false, true, false><<<ntiles, TILE_PX, 0, s>>>(a, g, dL_drgb, dL_dT, final_T, g_rec);
        raster_bwd_kernel<false, false, false><<<later, TILE_PX, 0, s>>>(a, g, dL_drgb, dL_dT, final_T, g_rec);
    }
    note_launches(2);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- K7: chain to the scene parameters


__global__ void __launch_bounds__(256) backward_params_kernel(CamParams c, SceneParams sp,
                                                              const float *__restrict__ g_rec,
                                                              const uint8_t *__restrict__ gflag,
                                                              float *__restrict__ g_means, float *__restrict__ g_ls,
                                                              float *__restrict__ g_quats,
                                                              float *__restrict__ g_logits, float *__restrict__ g_sh) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= sp.n || gflag[i] == 0) return;
    const float *gr = g_rec + 16 * i;
    bool any = false;
#pragma unroll
    for (int k = 0; k < 16; ++k) any |= gr[k] != 0.0f;
    if (!any) return;
    const float mu[3] = {sp.means[3 * i], sp.means[3 * i + 1], sp.means[3 * i + 2]};
    const float v[3] = {mu[0] - c.o[0], mu[1] - c.o[1], mu[2] - c.o[2]};   // mu - o
    const float L = sqrtf(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
    // quaternion, rotation, scales
    const float qr[4] = {sp.quats[4 * i], sp.quats[4 * i + 1], sp.quats[4 * i + 2], sp.quats[4 * i + 3]};
    const float qn = sqrtf(qr[0] * qr[0] + qr[1] * qr[1] + qr[2] * qr[2] + qr[3] * qr[3]);
    const float w = qr[0] / qn, x = qr[1] / qn, y = qr[2] / qn, z = qr[3] / qn;
    const float R[9] = {1.f - 2.f * (y * y + z * z), 2.f * (x * y - w * z), 2.f * (x * z + w * y),
                        2.f * (x * y + w * z), 1.f - 2.f * (x * x + z * z), 2.f * (y * z - w * x),
                        2.f * (x * z - w * y), 2.f * (y * z + w * x), 1.f - 2.f * (x * x + y * y)};
    const float rho2 = sp.rho2 ? sp.rho2[i] : 0.0f;
    float s[3], seff[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        s[a] = expf(sp.log_scales[3 * i + a]);
        seff[a] = sqrtf(s[a] * s[a] + rho2);
    }
    const float logit = load_scalar(sp.logits, i, sp.storage);
    const float sig = 1.0f / (1.0f + expf(-logit));
    const float sig_eff = sp.sig_eff[i];
    // dL/dW including o_u = W (o - mu); dL/dmu from o_u
    float gW[9];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) gW[3 * a + b] = gr[3 * a + b] + gr[9 + a] * (-v[b]);
    float gmu[3] = {0.f, 0.f, 0.f};
    const float *Wm = sp.W + 9 * i;
#pragma unroll
    for (int b = 0; b < 3; ++b) gmu[b] = -(Wm[b] * gr[9] + Wm[3 + b] * gr[10] + Wm[6 + b] * gr[11]);
    // W_ab = R_ba / seff_a
    float gR[9] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f}, gseff[3] = {0.f, 0.f, 0.f};
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            gR[3 * b + a] += gW[3 * a + b] / seff[a];
            gseff[a] += -gW[3 * a + b] * R[3 * b + a] / (seff[a] * seff[a]);
        }
    // sigma_eff = sigma prod s/seff
    const float gsig_eff = gr[12];
    float gls[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const float gs = gseff[a] * s[a] / seff[a] + gsig_eff * sig_eff * (1.0f / s[a] - s[a] / (seff[a] * seff[a]));
        gls[a] = gs * s[a];
    }
    const float gsig = sig > 0.0f ? gsig_eff * sig_eff / sig : 0.0f;
    const float glogit = gsig * sig * (1.0f - sig);
    // R(q/|q|)
    const float gw = 2.f * (-z * gR[1] + y * gR[2] + z * gR[3] - x * gR[5] - y * gR[6] + x * gR[7]);
    const float gx = 2.f * (y * gR[1] + z * gR[2] + y * gR[3] - 2.f * x * gR[4] - w * gR[5] + z * gR[6] +
                            w * gR[7] - 2.f * x * gR[8]);
    const float gy = 2.f * (-2.f * y * gR[0] + x * gR[1] + w * gR[2] + x * gR[3] + z * gR[5] - w * gR[6] +
                            z * gR[7] - 2.f * y * gR[8]);
    const float gz = 2.f * (-2.f * z * gR[0] - w * gR[1] + x * gR[2] + w * gR[3] - 2.f * z * gR[4] + y * gR[5] +
                            x * gR[6] + y * gR[7]);
    const float dotq = w * gw + x * gx + y * gy + z * gz;
    const float gqn[4] = {(gw - w * dotq) / qn, (gx - x * dotq) / qn, (gy - y * dotq) / qn, (gz - z * dotq) / qn};
    // colour: rgb = max(0, SH(u) + 1/2), u = (mu - o)/L
    const int K = (sp.sh_degree + 1) * (sp.sh_degree + 1);
    float u[3] = {0.f, 0.f, 1.f};
    if (L > 0.0f) { u[0] = v[0] / L; u[1] = v[1] / L; u[2] = v[2] / L; }
    float gu[3] = {0.f, 0.f, 0.f};
    float act[3];                  // dL/drgb of the channels above the max(0, .) clamp
    bool any_col = false;
#pragma unroll
    for (int ch = 0; ch < 3; ++ch) any_col |= gr[13 + ch] != 0.0f;
    if (any_col) {
        float Y[16], shc[48];
        sh_basis(u[0], u[1], u[2], sp.sh_degree, Y);
        load_sh(sp.sh, i, K, sp.storage, shc);
#pragma unroll
        for (int ch = 0; ch < 3; ++ch) {
            float raw = 0.5f;
#pragma unroll
            for (int j = 0; j < 16; ++j)
                if (j < K) raw += shc[3 * j + ch] * Y[j];
            act[ch] = raw > 0.0f ? gr[13 + ch] : 0.0f;
        }
        // dL/du = sum_j (sum_ch act_ch c_j,ch) dY_j/du
        float wj[16];
#pragma unroll
        for (int j = 0; j < 16; ++j)
            wj[j] = j < K ? act[0] * shc[3 * j] + act[1] * shc[3 * j + 1] + act[2] * shc[3 * j + 2] : 0.0f;
        sh_basis_grad_acc(u[0], u[1], u[2], sp.sh_degree, wj, gu);
        if (g_sh && (act[0] != 0.0f || act[1] != 0.0f || act[2] != 0.0f)) {
            float *gs = g_sh + (size_t)3 * K * i;
            if (((3 * K) & 3) == 0) {            // float4 read-modify-write (degrees 1 and 3)
                float4 *g4 = reinterpret_cast<float4 *>(gs);
#pragma unroll
                for (int q = 0; q < 12; ++q) {
                    if (4 * q < 3 * K) {
                        float4 v = g4[q];
                        const int e = 4 * q;
                        v.x += act[(e) % 3] * Y[(e) / 3];
                        v.y += act[(e + 1) % 3] * Y[(e + 1) / 3];
                        v.z += act[(e + 2) % 3] * Y[(e + 2) / 3];
                        v.w += act[(e + 3) % 3] * Y[(e + 3) / 3];
                        g4[q] = v;
                    }
                }
            } else {
#pragma unroll
                for (int j = 0; j < 16; ++j)
                    if (j < K) {
                        gs[3 * j] += act[0] * Y[j];
                        gs[3 * j + 1] += act[1] * Y[j];
                        gs[3 * j + 2] += act[2] * Y[j];
                    }
            }
        }
    }
    if (L > 0.0f) {
        const float ud = u[0] * gu[0] + u[1] * gu[1] + u[2] * gu[2];
#pragma unroll
        for (int k = 0; k < 3; ++k) gmu[k] += (gu[k] - u[k] * ud) / L;
    }
    if (g_means) {
#pragma unroll
        for (int k = 0; k < 3; ++k) g_means[3 * i + k] += gmu[k];
    }
    if (g_ls) {
#pragma unroll
        for (int k = 0; k < 3; ++k) g_ls[3 * i + k] += gls[k];
    }
    if (g_quats) {
#pragma unroll
        for (int k = 0; k < 4; ++k) g_quats[4 * i + k] += gqn[k];
    }
    if (g_logits) g_logits[i] += glogit;
}

cudaError_t launch_backward_params(const CamParams &c, const SceneParams &sp, const float *g_rec,
                                   const uint8_t *gflag, const float4 *gview, float *g_means, float *g_log_scales,
                                   float *g_quats, float *g_logits, float *g_sh, cudaStream_t s) {
    (void)gview;
    if (sp.n == 0) return cudaSuccess;
    backward_params_kernel<<<(unsigned)div_up(sp.n, 256), 256, 0, s>>>(c, sp, g_rec, gflag, g_means, g_log_scales,
                                                                      g_quats, g_logits, g_sh);
    note_launches(1);
    return cudaGetLastError();
}

}  // namespace conegs
